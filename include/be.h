/*
 * be.h -- C ABI of the B300 batched-einsum engine.
 *
 * A batched einsum (b, n, I_out, (I_in,j)_j, ((A^{i,j})_j)_i) is b einsums
 * that share one Einstein notation and may share operands (paper, Sec.
 * "Batched Einstein Summation", Def. of a batched einsum).  Its operands may
 * be lambdas over buffers (Sec. "Integration of Optimized Batched Einsums
 * into Practical Programs", Def. "Functional Batched Einstein Summation").
 * The engine parses such a spec, maps it to a normal form (Sec. "A
 * Canonical form for Batched Einsums", Alg. 1), looks a tuned configuration
 * up under that form and transfers it to the caller's names (Alg. 2), and
 * evaluates the batch on the GPU (Eq. (1) per row).
 *
 * Conventions for every call:
 *   - Return value: BE_OK (0) or one of the BE_E* codes below.  No C++
 *     exception crosses this boundary.  be_last_error() gives a message for
 *     the calling thread's last failure.
 *   - Handles (be_einsum, be_canon, be_ctx) are allocated by the library
 *     and released by the matching be_free_* / be_ctx_destroy.
 *   - Device memory passed in be_buf is owned by the caller and only
 *     borrowed for the duration of the (asynchronous) work on the stream.
 *   - Strings written into caller buffers are NUL-terminated; when the
 *     buffer is too small the call writes nothing, stores the needed size
 *     (including the NUL) in *needed and returns BE_EARG.
 */
#ifndef BE_H
#define BE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define BE_OK 0
#define BE_EPARSE 1        /* text does not follow the grammar of be_parse        */
#define BE_EINVALID 2      /* violates a soundness rule of Eq. (1) (Sec. "Preliminaries") */
#define BE_ESHAPE 3        /* inconsistent axis lengths / buffer shapes           */
#define BE_EDTYPE 4        /* unknown or mismatching dtype                        */
#define BE_ETOOMANY 5      /* beyond a stated limit (26 indices, 16 operands ...) */
#define BE_ENOTFOUND 6     /* no tuning record under this normal form             */
#define BE_EDB 7           /* tuning database file unreadable or corrupt          */
#define BE_EBUDGET 8       /* request does not fit the HBM admission budget       */
#define BE_ETIMEOUT 9      /* a bounded device-side wait ran out                  */
#define BE_ECUDA 10        /* a CUDA runtime call failed                          */
#define BE_EUNSUPPORTED 11 /* valid input the engine does not handle              */
#define BE_EARG 12         /* bad argument (NULL handle, buffer too small, ...)   */

/* ---- dtypes: the DtypeRank values of the induced-graph appendix; bfloat16 = 9 ---- */
#define BE_I8 1
#define BE_I32 2
#define BE_I64 3
#define BE_F16 4
#define BE_F32 5
#define BE_F64 6
#define BE_C64 7
#define BE_C128 8
#define BE_BF16 9

/* ---- evaluation strategies (be_config.strategy) ---- */
#define BE_STRAT_AUTO 0        /* pick by pattern: ELEMENT, DENSE_SPLIT, else GENERIC   */
#define BE_STRAT_GENERIC 1     /* one thread per output element, any notation           */
#define BE_STRAT_ELEMENT 2     /* shared small operators x streamed per-element operands;
                                  tile[0] elements per tile, tile[1] threads per CTA,
                                  tile[2] variant (1 FP64 pipe, 2 double-float on the FP32
                                  pipe, 3 tensor-core digit split, also for the stacked
                                  divergence / face-mass form up to 64 contracted values;
                                  0 = tensor cores where the shape allows and the form is
                                  not stacked, else double-float), tile[3] for small
                                  operators (at most 8 x 8) on the double-float variant:
                                  1 + the share of the elements, in sixteenths, that run
                                  on the FP64 pipe beside the double-float ones (0 = 8/16) */
#define BE_STRAT_DENSE_SPLIT 3 /* FP64 contraction as products of three BF16 parts per
                                  operand on tcgen05 (FP32 accumulation, compensated
                                  drains); needs a context (its workspace holds the split
                                  operands); tile[2] k-blocks of 64 between drains of the
                                  leading-product accumulator (0 = 1, whose a-priori bound
                                  is within 1e-6; 2 and more are faster, with bounds of
                                  about 1.4e-6 and above); split >= 4 adds the next level's
                                  two products */

/* ---- precision modes (part of the tuning key, not of the normal form) ---- */
#define BE_PREC_FP64 0         /* results within 1e-12 of the absolute contraction */
#define BE_PREC_SPLIT 1        /* split-precision tensor-core products, within 1e-6 */

/* ---- sigma kinds for be_canon_sigma ---- */
#define BE_SIGMA_INDEX 0       /* canonical index letter k -> user index letter     */
#define BE_SIGMA_ARG 1         /* canonical argument A<k> -> user argument name     */
#define BE_SIGMA_ROW 2         /* canonical row k -> user row (decimal)             */
#define BE_SIGMA_POS 3         /* canonical operand position k -> user position     */

typedef struct be_ctx be_ctx;
typedef struct be_einsum be_einsum;
typedef struct be_canon be_canon;
typedef struct be_batch be_batch;
typedef struct be_server be_server;

/* A tuned configuration, stated on the canonical form's names. */
typedef struct {
  int32_t strategy;    /* BE_STRAT_*                                          */
  int32_t tile[4];     /* strategy tile sizes (0 = strategy default)          */
  int32_t stages;      /* pipeline depth (0 = default)                        */
  uint32_t stage_mask; /* bit k: keep canonical argument A<k> in shared memory */
  int32_t vec;         /* elements per vector access (0 = default)            */
  int32_t split;       /* split-precision product terms (0 = none)            */
} be_config;

/* A caller-owned array.  For be_execute ptr is a device pointer; for
 * be_execute_host a host pointer.  strides: elements per step of each
 * dimension (NULL: dense row-major).  dtype: BE_* above. */
typedef struct {
  void *ptr;
  const int64_t *strides;
  int32_t ndim;
  int32_t dtype;
} be_buf;

/* Library version (major*10000 + minor*100 + patch). */
int be_version(void);

/* Message of the calling thread's last failed call ("" if none). */
const char *be_last_error(void);

/*
 * be_parse -- text -> batched-einsum IR.
 *   text:  "<notation> | <row> | <row> ... ; <decl> ; <decl> ..."
 *          notation "ij,ej->ei" over letters a..z (Sec. "Preliminaries",
 *          index grammar); each row lists one argument name per operand;
 *          decl "name:dtype[d0,d1,..]" declares a buffer, and
 *          "name(p,q,..)[:dtype[dims]] := expr" a lambda operand whose body
 *          uses + - * / unary -, sin cos exp abs, numbers, $scalars,
 *          buffer refs name[p,0,..] and "p==k ? x : y".
 *   out:   new handle on success (free with be_free_einsum).
 * Errors: BE_EPARSE (grammar), BE_EINVALID (soundness: Dim vs index list,
 * output index not in any input, repeated output index, n = 0),
 * BE_ESHAPE (unequal lengths of one index), BE_EDTYPE, BE_ETOOMANY
 * (> 16 operands or > 4096 rows), BE_EUNSUPPORTED (0-dimensional operand).
 */
int be_parse(const char *text, be_einsum **out);
void be_free_einsum(be_einsum *e);

/* Sizes of a parsed einsum: rows b, operands n, declared buffers, distinct
 * idealized arguments, runtime scalars, output rank and output dtype. */
int be_einsum_info(const be_einsum *e, int32_t *b, int32_t *n, int32_t *n_buffers,
                   int32_t *n_args, int32_t *n_scalars, int32_t *out_ndim, int32_t *out_dtype);
/* Output shape (out_ndim entries). */
int be_einsum_out_shape(const be_einsum *e, int64_t *shape);
/* Declared buffer k (declaration order): name, dtype, rank and shape (up to 26 entries). */
int be_einsum_buffer(const be_einsum *e, int32_t k, char *name, size_t len, size_t *needed,
                     int32_t *dtype, int32_t *ndim, int64_t *shape);

/*
 * be_canonicalize -- Alg. 1: the normal form C(e) and the maps from its
 * symbols to e's (sigma^I, sigma^A, and the row / operand orders).
 * C(e) = C(e') iff e and e' are isomorphic batched einsums (Def. of a
 * canonicalization function); our C is the lexicographically smallest
 * token vector over operand and row orders with first-appearance naming.
 */
int be_canonicalize(const be_einsum *e, be_canon **out);
void be_free_canon(be_canon *c);
/* Printed normal form "be1:<b>;<n>;<out>-><ins>;<lengths>;<rows>;<dtypes>". */
int be_canon_key(const be_canon *c, char *buf, size_t len, size_t *needed);
/* Name in the user's einsum of canonical symbol canon_id of the given kind. */
int be_canon_sigma(const be_canon *c, int32_t kind, int32_t canon_id, char *user_name, size_t len,
                   size_t *needed);
/* Token vector of C(e) (for tests); count in *n_tokens. */
int be_canon_tokens(const be_canon *c, int64_t *tokens, size_t cap, size_t *n_tokens);

/*
 * Induced graph of Appendix B.1 (for tests).  colors: cap_nodes entries,
 * 1..9; edges: cap_edges (from, to) pairs.  Sizes go to *n_nodes / *n_edges.
 */
int be_induced_graph(const be_einsum *e, int32_t *n_nodes, int32_t *colors, int32_t cap_nodes,
                     int32_t *edges, int64_t cap_edges, int64_t *n_edges);
/* Compliance conditions of Appendix B.2 on a caller graph: *failed = 0 if
 * all hold, else the number k of the first failing condition (Ck). */
int be_graph_check(int32_t n_nodes, const int32_t *colors, const int32_t *edges, int64_t n_edges,
                   int32_t *failed);

/*
 * be_identify -- Alg. 2: express a stored reference einsum's names in a
 * target einsum's names.  Both are canonicalized; if the normal forms
 * differ the call returns BE_EINVALID (the algorithm's exception).
 * Otherwise writes "ref=target;..." pairs for every index (letters) and
 * argument (names) of ref.
 */
int be_identify(const be_einsum *ref, const be_einsum *target, char *buf, size_t len, size_t *needed);

/*
 * be_raise -- RaiseToBatchedEinsum, the first step of Alg. 2 (Sec.
 * "Integration with other frameworks"): read a loop-nest kernel back as
 * the functional batched einsum it computes.  kernel: lines of
 *   "{ [i0,i1,..] : 0<=i0<N0 and 0<=i1<N1 .. }"   loop domain
 *   "name:dtype[d0,d1,..]"                         input array
 *   "name(p,q,..) := expr"                         substitution rule (expr as in be_parse)
 *   "for i0" ... "end"                             loop nesting
 *   "y[i0,..] = sum([i1,..], f(..)*g(..)*..)"      statement (or a plain product)
 * ('#' starts a comment).  A factor is a rule call r(i0,..) or an array
 * access A[i0,..] with loop names as subscripts; output subscripts are
 * enclosing loops, the others are summed.  Each statement is one row; all
 * rows must share one index structure up to a renaming of their loop names
 * and the order of their factors.  Index letters are the loop names of the
 * first statement in order of first appearance (output, then factors).
 *   out: new handle (free with be_free_einsum), usable wherever a parsed
 *        einsum is: canonicalize, lookup, identify, execute (one buffer per
 *        declared array, declaration order).
 * Errors: BE_EPARSE (kernel grammar), BE_EINVALID (unknown names, bad
 * subscripts, statements that do not form one batched einsum), BE_ETOOMANY
 * (> 26 loop indices), and the errors of be_parse on the raised text.
 */
int be_raise(const char *kernel, be_einsum **out);

/*
 * be_record_facts -- record_facts of the transformation writer's view (Sec.
 * "Integration with other frameworks"): time cfg on the idealized reference
 * einsum ref -- device operands of its declared shapes filled with
 * synthetic values (floating types uniform in [-1, 1), integers -3..3),
 * every runtime scalar 1 -- after `warmup` untimed runs, average `reps`
 * timed runs (CUDA events on the default stream), and store the time with
 * be_record under ref's normal form.  The library allocates and frees the
 * synthetic operands itself.  *seconds (may be NULL) receives the time.
 * Errors: BE_EARG, the errors of be_execute for a cfg that does not fit ref,
 * BE_ECUDA (allocation, launch), BE_EDB.
 */
int be_record_facts(be_ctx *x, const be_einsum *ref, const be_config *cfg, int32_t precision, int32_t warmup,
                    int32_t reps, double *seconds);

/*
 * be_load_transforms -- a user-supplied transform library: one registration
 * per line, "<reference in be_parse text> => <strategy> <tile0> <tile1>
 * <tile2> <tile3> [<stages> <stage_mask> <vec> <split> [<precision>]]"
 * ('#' starts a comment line).  Every line is parsed first (BE_EPARSE or the
 * be_parse error of the reference, with its line number, and nothing is
 * timed); then each is recorded with be_record_facts.  *n_recorded (may be
 * NULL) counts the registrations stored.
 */
int be_load_transforms(be_ctx *x, const char *text, int32_t warmup, int32_t reps, int32_t *n_recorded);

#define BE_RAISED_SPEC 0     /* the be_parse text the kernel was raised to       */
#define BE_RAISED_LOOP 1     /* k: loop name of index letter 'a' + k            */
#define BE_RAISED_OUTPUT 2   /* k: output array of row k                         */
/* Names kept by be_raise (BE_ENOTFOUND for an einsum that was parsed, or
 * k out of range); the string goes to buf like the other string calls. */
int be_raised_name(const be_einsum *e, int32_t kind, int32_t k, char *buf, size_t len, size_t *needed);

/*
 * Tuning database keyed by (normal form, device name, precision mode),
 * the paper's database of performance facts (Introduction, Fig. "The
 * Feinsum approach").  db_path: append-only text file, created if missing;
 * NULL keeps the database in memory.  device_name: the key's device field;
 * NULL uses the CUDA name of `device`.  hbm_budget_bytes bounds device
 * memory admitted by the serving loop (0 = unbounded).
 * Errors: BE_EDB when the file exists but a record is malformed.
 */
int be_ctx_create(const char *db_path, const char *device_name, int32_t device,
                  size_t hbm_budget_bytes, be_ctx **out);
void be_ctx_destroy(be_ctx *x);
/* Best stored config for c's normal form (BE_ENOTFOUND if none). */
int be_lookup(be_ctx *x, const be_canon *c, int32_t precision, be_config *out, double *seconds);
/* Store a measured config (appended to the file); the best per key wins. */
int be_record(be_ctx *x, const be_canon *c, int32_t precision, const be_config *cfg, double seconds);
/* Number of distinct keys held. */
int be_db_size(be_ctx *x, int64_t *n);

/*
 * be_execute -- evaluate every row of e on `stream` (cudaStream_t; NULL =
 * default stream), asynchronously.
 *   bufs:    one be_buf per declared buffer of e, declaration order, device
 *            pointers, dtype equal to the declaration; strides may be NULL.
 *   outs:    one dense row-major device array per row (output shape, dtype
 *            e's output dtype = highest-ranked argument dtype).
 *   scalars: values of e's runtime scalars ($name), first-appearance order.
 *   cfg:     NULL looks the config up in x's database under the normal form
 *            and precision; without a record the strategy's defaults run.
 * Errors: BE_EARG / BE_EDTYPE / BE_ESHAPE for mismatching buffers,
 * BE_EUNSUPPORTED when a forced strategy does not fit e, BE_ECUDA.
 */
int be_execute(be_ctx *x, const be_einsum *e, const be_config *cfg, int32_t precision,
               const be_buf *bufs, int32_t n_bufs, const be_buf *outs, int32_t n_outs,
               const double *scalars, int32_t n_scalars, void *stream);

/*
 * be_execute_host -- as be_execute with HOST buffers: copies the inputs to
 * device memory owned by x, evaluates, copies the outputs back and waits
 * for the stream.  The staging memory is kept in x and reused.
 */
int be_execute_host(be_ctx *x, const be_einsum *e, const be_config *cfg, int32_t precision,
                    const be_buf *bufs, int32_t n_bufs, const be_buf *outs, int32_t n_outs,
                    const double *scalars, int32_t n_scalars, void *stream);

/*
 * be_tune -- the autotuner that fills the database (the paper's transform
 * writer recording performance facts under the normal form, Sec.
 * "Integration of Optimized Batched Einsums into Practical Programs").
 * Every configuration of every strategy that fits e and `precision` is run
 * `warmup` times, then timed with CUDA events on `stream` until at least
 * `min_reps` runs and `min_seconds` of kernel time (the paper's protocol is
 * warmup = 5, min_reps = 20, min_seconds = 2); each mean is recorded with
 * be_record under C(e), and the fastest is returned in *best.  With force = 0
 * a key already in the database is returned without timing (resume).
 * The outputs are overwritten while timing.  *n_tried counts timed configs.
 */
int be_tune(be_ctx *x, const be_einsum *e, int32_t precision, const be_buf *bufs, int32_t n_bufs,
            const be_buf *outs, int32_t n_outs, const double *scalars, int32_t n_scalars, int32_t warmup,
            int32_t min_reps, double min_seconds, int32_t force, void *stream, be_config *best,
            double *best_seconds, int32_t *n_tried);

/*
 * Persistent multi-instance executor: many batched einsums (any notations,
 * sizes and dtypes) evaluated by ONE persistent launch, replayed as a CUDA
 * graph.  The batched einsum is the paper's primitive (Sec. "Batched
 * Einstein Summation"); grouping several of them into one launch removes
 * the per-launch overhead that dominates small einsums.
 *
 * be_batch_create -- plan n instances: es[k] with its declared buffers
 *   bufs[k][0..n_bufs[k]) and outputs outs[k][0..n_outs[k]) (device
 *   pointers, as for be_execute) and runtime scalars scalars[k] (may be
 *   NULL when n_scalars is NULL or 0).  Each instance gets a strategy:
 *   element-shaped FP64 instances (shared small operator, streamed
 *   per-element operands) take the element strategy with their database
 *   configuration (cfg->stage_mask bit 0 keeps them generic); with
 *   cfg->split >= 1, FP64 instances of GEMM form with at least
 *   2^cfg->tile[3] multiply-adds (default 2^23) take the split-precision
 *   tensor-core strategy (1e-6 * S); every other instance is generic: each
 *   of its rows becomes a descriptor whose outputs are cut into tiles of
 *   about 2^tile[1] operand terms (default 20) for one persistent launch
 *   (cfg->tile[0] its block size, default 256, and 256 whenever a row is
 *   evaluated as GEMM tiles; cfg->tile[2] CTAs per SM, default 4).  A
 *   generic instance of 2 to 5 operands, all views of buffers, whose best
 *   order of steps (fewest multiply-adds over all orders of two-operand
 *   contractions and of one-operand sums of an operand's own letters) cuts the multiply-adds of Eq. (1)'s loop nest at least
 *   1.5 times is factored: each row runs as that sequence of two-operand
 *   einsums over dense intermediates (the same sum with its terms grouped
 *   differently); a step's tiles follow the tiles of the steps it reads in
 *   the one persistent launch and wait (bounded) until those have finished,
 *   the intermediates in a workspace owned by the batch
 *   (cfg->stage_mask bit 1 keeps every instance on its loop nest).  With
 *   cfg->split >= 2 a factored FP64 instance of two steps whose last step
 *   is a GEMM of at least 2^tile[3] multiply-adds (the output's letters
 *   those of the first step's result and then those of one operand, or the
 *   reverse), carrying at least half of its multiply-adds, runs on a dense
 *   branch instead: per row the first step (and, when the operand's own
 *   layout does not flatten to the GEMM, a permuted copy of it) as generic
 *   launches, then the split-precision GEMM (1e-6 * S).  cfg may
 *   be NULL.  Everything is captured once in a CUDA
 *   graph with concurrent branches: the persistent launch of generic
 *   tiles, the element launches and the split / GEMM launches (four
 *   branches, each with a split workspace owned by the batch).  The element and dense launches
 *   run once during creation.  The buffers are borrowed and must stay valid
 *   while the batch is used; their CONTENTS may change between runs.
 *   Device memory for descriptors, tiles and the workspace is allocated
 *   here.
 * be_batch_run -- replay the captured graph on `stream` (asynchronous).
 *   Every output has a single owner and a fixed evaluation order, so the
 *   results are bitwise those of be_execute on each instance alone with
 *   the strategy it was given (BE_STRAT_GENERIC for generic instances),
 *   except factored instances, whose grouping of the terms differs (within
 *   the precision mode's tolerance) and is itself deterministic.
 * be_batch_info -- rows, tiles and total operand terms of the generic part
 *   (factored steps counted as rows).
 * be_batch_kinds -- number of instances given each strategy (the
 *   dense-routed factored instances count as dense).
 * be_batch_instance_kind -- the evaluation of instance k: 0 generic loop
 *   nest, 1 element, 2 dense (split precision), 3 factored steps in the
 *   persistent launch, 4 factored steps on a dense branch (split precision);
 *   BE_EARG for k outside 0 .. n - 1.
 * be_batch_factored -- number of factored instances in the persistent
 *   launch, the longest chain of dependent steps (phases; 1 without
 *   factored instances), and bytes of the intermediates' workspace.
 */
int be_batch_create(be_ctx *x, int32_t n, const be_einsum *const *es, const be_buf *const *bufs,
                    const int32_t *n_bufs, const be_buf *const *outs, const int32_t *n_outs,
                    const double *const *scalars, const int32_t *n_scalars, const be_config *cfg,
                    be_batch **out);
int be_batch_run(be_batch *b, void *stream);
int be_batch_info(const be_batch *b, int64_t *rows, int64_t *tiles, double *terms);
int be_batch_kinds(const be_batch *b, int32_t *generic, int32_t *element, int32_t *dense);
int be_batch_instance_kind(const be_batch *b, int32_t k, int32_t *kind);
int be_batch_factored(const be_batch *b, int32_t *instances, int32_t *phases, int64_t *workspace_bytes);

/*
 * be_tune_batch -- the autotuner for a batch (tile shapes and schedules
 * chosen by the engine's own tuner, results kept in the database beside
 * the normal-form keys, Sec. "Integration..." performance facts).  Creates the batch of be_batch_create
 * under each candidate launch shape of its persistent part -- block size
 * 128 (skipped when a row is evaluated as GEMM tiles) or 256, 2, 3 or 4 CTAs
 * per SM, tiles of 2^18, 2^20 or 2^22 operand terms -- with base's strategy policy (split, tile[3], stage_mask; base
 * may be NULL), times reps graph replays on `stream` after one warm-up, and
 * records every timed candidate in x's database under the batch key: the
 * instances' canonical keys, sorted and hashed, so any renaming or
 * reordering of the same instances finds the record.  be_batch_create with
 * cfg == NULL then uses the best record.  Returns the best configuration,
 * its seconds per replay and the number of candidates timed.  The element
 * and dense launches of the batch run once per candidate.  Errors:
 * BE_EARG, BE_EDB, BE_EUNSUPPORTED (no candidate ran), BE_ECUDA.
 */
int be_tune_batch(be_ctx *x, int32_t n, const be_einsum *const *es, const be_buf *const *bufs,
                  const int32_t *n_bufs, const be_buf *const *outs, const int32_t *n_outs,
                  const double *const *scalars, const int32_t *n_scalars, const be_config *base, int32_t reps,
                  void *stream, be_config *best, double *best_seconds, int32_t *n_tried);
void be_batch_destroy(be_batch *b);

/*
 * Serving loop with continuous batching.  Requests are parsed batched
 * einsums whose buffers and outputs are already on the device.
 * be_server_create -- a worker thread plus n_streams CUDA streams on the
 *   current device; requests run in `precision` with the configuration
 *   stored under their normal form in x's database (memoized by text).
 *   hbm_budget_bytes (0: x's budget; 0 there too: unbounded) caps the bytes
 *   that requests in flight may pin (their declared buffers and outputs).
 * be_server_submit -- queue a request (asynchronous; returns an id).  The
 *   einsum handle and the buffers must stay valid until the request is done.
 *   Requests are admitted in arrival order while the budget allows and are
 *   launched at once on the next stream, so they overlap on the device with
 *   requests already running; a request larger than the whole budget
 *   finishes with status BE_EBUDGET.  Split-precision requests share the
 *   context's workspace and therefore run on one stream.
 * be_server_wait -- block until request id is done (timeout_s < 0: no
 *   limit; BE_ETIMEOUT otherwise), return its status and latency (submit to
 *   completion of its last kernel), and forget it.
 * be_server_drain -- block until nothing is queued or running.
 * be_server_stats -- completed / failed counts, p50 / p99 latency,
 *   throughput (completed / span from first submit to last completion), peak
 *   bytes and peak number of requests in flight.
 */
int be_server_create(be_ctx *x, int32_t precision, int32_t n_streams, size_t hbm_budget_bytes, be_server **out);
int be_server_submit(be_server *s, const be_einsum *e, const be_buf *bufs, int32_t n_bufs, const be_buf *outs,
                     int32_t n_outs, const double *scalars, int32_t n_scalars, int64_t *id);
int be_server_wait(be_server *s, int64_t id, double timeout_s, int32_t *status, double *latency_s);
int be_server_drain(be_server *s, double timeout_s);
int be_server_stats(be_server *s, int64_t *completed, int64_t *failed, double *p50_s, double *p99_s,
                    double *throughput, size_t *peak_bytes, int64_t *max_inflight);
int be_server_reset_stats(be_server *s);
/*
 * be_server_trace -- the tracing view of the requests completed since the
 * last reset: per request six doubles (id, submit, admit, launched, done,
 * stream index), times in seconds of a steady clock; `launched` is when
 * the request's launch calls returned on the worker thread, `done` when
 * the completion thread saw its event.  Copies min(cap, n) rows into rows
 * (6 doubles each, completion order) and returns n.  Errors: BE_EARG.
 */
int be_server_trace(be_server *s, double *rows, int64_t cap, int64_t *n);
void be_server_destroy(be_server *s);

/*
 * be_status -- wait for the device, then read and clear x's device status
 * word: BE_OK, or BE_ETIMEOUT when a bounded device-side wait of a kernel
 * launched through x ran out (the kernel then stopped early and its output
 * is not valid).
 */
int be_status(be_ctx *x, int32_t *device_status);

/*
 * be_ctx_set_wait_limit -- limit, in SM clock cycles, of every pipeline
 * wait of the tensor-core kernels (the element strategy's digit-split GEMM
 * and the dense split GEMM) launched through x, and of the dependency waits
 * of factored steps in batches created with x (the limit in force when the
 * batch is created); 0 restores the default of about one second.  A wait that runs out stops its kernel early (outputs
 * not valid), frees the kernel's tensor memory after its issued work has
 * completed, and leaves BE_ETIMEOUT for be_status.  A limit of a few
 * thousand cycles makes the waits run out on purpose (failure-path tests);
 * the paper has no counterpart.  Errors: BE_EARG.
 */
int be_ctx_set_wait_limit(be_ctx *x, int64_t cycles);

/* ---- per-kernel timing (CUDA events on the launching stream) ---- */
#define BE_KERNEL_ELEMENT 0     /* element-streaming kernel              */
#define BE_KERNEL_GENERIC 1     /* generic loop-nest kernel              */
#define BE_KERNEL_DENSE_GEMM 2  /* tcgen05 split-precision GEMM          */
#define BE_KERNEL_SPLIT 3       /* operand split kernels of that strategy */
#define BE_KERNEL_PERSISTENT 4  /* persistent multi-instance executor    */

/* Enable (1) or disable (0) event timing of every kernel launched through x. */
int be_ctx_set_timing(be_ctx *x, int32_t enable);
/* Wait for, sum and forget the recorded launches of one kernel id. */
int be_ctx_timing(be_ctx *x, int32_t kernel, int64_t *launches, double *total_ms);

/*
 * be_gemm_split_noalloc -- C = A * B for FP64 row-major matrices (A: M x K,
 * row stride lda; B: K x N, row stride ldb; C: M x N, row stride ldc) on the
 * split-precision tensor-core path of BE_STRAT_DENSE_SPLIT (same kernels,
 * same accuracy), asynchronously on `stream`, WITHOUT allocating any device
 * memory.  The paper has no counterpart to this call; it exists for callers
 * that cannot let a library allocate: applications that keep all device
 * memory in their own pool or budget, where a cudaMalloc inside a library
 * could fail or go unaccounted and a cudaFree could synchronize the device
 * and stall their other streams.
 *
 * Scratch: a fixed 64 MiB array compiled into the library (plus one status
 * word), held on every GPU where the library's device code is loaded until
 * the process exits.  With CUDA's default lazy module loading the driver
 * reserves the array on a device only when the first call there looks up
 * its address, so that first call (a warm-up) is where the 64 MiB are
 * taken, and it can fail with BE_ECUDA if the device is already full: make
 * it before the caller sets up its memory pool and before any stream
 * capture.  The call fails with BE_ETOOMANY (nothing launched) when the
 * problem needs more: about (M + N) * K * 6 bytes with M and N padded to
 * 128 and K to 64 (e.g. M = N = 1024, K = 5440 fits).  Every call reuses the
 * same array (the call clears what must start at zero), so calls whose GPU
 * work overlaps -- on different streams or devices sharing a context -- race;
 * issue them in order on one stream.  Errors: BE_EARG, BE_ETOOMANY,
 * BE_ECUDA, message in be_last_error().  A kernel whose bounded wait ran
 * out leaves BE_ETIMEOUT in the array's status word; read it with
 * be_gemm_split_noalloc_status.
 */
int be_gemm_split_noalloc(const double *A, int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc,
                          int64_t M, int64_t N, int64_t K, void *stream);

/*
 * be_gemm_split_noalloc_status -- read and clear the status word of the
 * current device's fixed array: BE_OK, or BE_ETIMEOUT when a call since the
 * last read stopped early (its C is then not valid).  Allocates nothing; it
 * copies one word synchronously with the device, so call it after the
 * stream that ran the calls has been synchronized.  The paper has no
 * counterpart.  Errors: BE_EARG, BE_ECUDA.
 */
int be_gemm_split_noalloc_status(int32_t *status);

/*
 * be_peak_probe -- measured peak rate of one pipe on the current device, in
 * TFLOP/s (2 flops per fused multiply-add): kind 0 FP64, kind 1 FP32.
 * Independent FMA chains in registers, no memory traffic; best of reps
 * timed launches after one warm-up.  The rooflines of the FP64 and
 * double-float evaluation paths are stated against these rates.  Allocates
 * a small output buffer.  Errors: BE_EARG, BE_ECUDA.
 */
int be_peak_probe(int32_t kind, int32_t reps, double *tflops);

/* Strategy the engine would run for e under cfg (after AUTO resolution). */
int be_plan_strategy(be_ctx *x, const be_einsum *e, const be_config *cfg, int32_t precision,
                     int32_t *strategy);

#ifdef __cplusplus
}
#endif

#endif /* BE_H */
