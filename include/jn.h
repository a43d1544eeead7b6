/*
 * jn.h -- GPU joins over integer key columns (GB300, sm_103a).
 *
 * C ABI of libjn.so.  It follows the paper's statement of the problem
 * (H. Wang et al., "GPU-based Efficient Join Algorithms on Hadoop",
 * arXiv 1904.11201):
 *   - a table arrives as column buffers in one row order, and a match of row
 *     m of R with row n of S yields the pair (m, n) -- here (payload_R[m],
 *     payload_S[n]) -- (Sec. 3.2.2, row and column transformation);
 *   - the GPU entry points take the two tables and their sizes, as
 *     Join_GPU(T', S', NB_T, NB_S) of Algorithm 1 and GPU_theta_join(S, T) of
 *     Algorithm 3 do;
 *   - the output is sized exactly by a count pass before it is written, in
 *     place of the Cartesian-product bound of Eq. (rsize) (Sec. 3.3.3).
 * R is the build side (the paper's T, "the smaller table", Sec. 2.3) and S the
 * probe side.
 *
 * General rules for every entry point:
 *   - Errors are returned as jn_status; nothing throws or aborts.  A CUDA
 *     error maps to JN_ERR_CUDA and jn_last_error() gives its text.
 *   - Column pointers may be device memory or host memory (pinned or
 *     pageable).  Host columns are copied to device scratch owned by the
 *     context before the join; device columns are read in place.  The caller
 *     keeps every column valid and unchanged until the call returns.
 *   - All work runs on the context's stream, in stream order.  Calls that
 *     size an output (jn_count, jn_aggregate and the three joins) read the
 *     8-byte count back to the host and therefore synchronise that stream.
 *   - A context is used by one host thread at a time.
 *   - Row counts are limited to 2^31 - 1 per table (JN_ERR_INVALID beyond).
 *   - Output order is unspecified; the multiset of pairs is exact.
 */
#ifndef JN_H
#define JN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    JN_OK = 0,
    JN_ERR_INVALID = 1,      /* bad argument: NULL pointer, key type mismatch, n out of range */
    JN_ERR_OOM = 2,          /* device allocation failed */
    JN_ERR_CAPACITY = 3,     /* caller buffer too small: *n_out = required pairs, nothing written */
    JN_ERR_CUDA = 4,         /* a CUDA call failed (see jn_last_error) */
    JN_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out */
    JN_ERR_UNSUPPORTED = 6   /* predicate or mode not implemented for this algorithm */
} jn_status;

typedef enum { JN_KEY_I32 = 4, JN_KEY_I64 = 8 } jn_key_type;

/* R.col op S.col.  Sec. 2.3 names =, >, <, >=, <= "and so on"; Sec. 4.2's
 * region figure adds !=.  JN_ANY is the always-true predicate. */
typedef enum {
    JN_EQ = 0, JN_NE = 1, JN_LT = 2, JN_LE = 3, JN_GT = 4, JN_GE = 5, JN_ANY = 6
} jn_op;

typedef enum { JN_ALGO_NLJ = 0, JN_ALGO_HASH = 1, JN_ALGO_THETA = 2, JN_ALGO_SORT = 3 } jn_algo;

/* One table as column buffers (Sec. 3.2.2).  Signed integers; all key columns
 * of one call share key_type. */
typedef struct {
    const void* key;          /* n values: the join column (theta: column a)            */
    const void* key2;         /* n values: second compared column (band: column k), or NULL */
    const int32_t* payload;   /* n int32 values emitted in the pairs, or NULL = row index */
    int64_t n;                /* rows, 0 .. 2^31-1                                       */
    int32_t key_type;         /* JN_KEY_I32 or JN_KEY_I64                                */
    int32_t reserved;         /* must be 0                                               */
} jn_table;

/* One result: (R.payload[m], S.payload[n]); (m, n) when payloads are NULL. */
typedef struct {
    int32_t r;
    int32_t s;
} jn_pair;

/* One result of a star join: (R.payload[m], S1.payload[n1], S2.payload[n2]);
 * row indices when a payload column is NULL. */
typedef struct {
    int32_t r;
    int32_t s1;
    int32_t s2;
} jn_triple;

/* Two-column conjunctive predicate:
 *     (R.key op_a S.key) AND (band >= 0 ? |R.key2 - S.key2| <= band
 *                                       : R.key2 op_k S.key2)
 * The second conjunct is dropped (true) when either key2 is NULL.  |R.key2 -
 * S.key2| is evaluated exactly (no overflow).  NULL pred = equality on key. */
typedef struct {
    int32_t op_a;
    int32_t op_k;
    int64_t band;
} jn_pred;

/* Tuning knobs; 0 (or -1 where noted) lets the library choose.  The result
 * never depends on them. */
typedef struct {
    int32_t prefilter;     /* Algorithm 1's common-key filter: -1 auto, 0 off, 1 both
                              tables, 2 only S (by R's keys), 3 only R (by S's keys).
                              Auto: off below 2^22 rows in all; else only the larger
                              table when it has twice the other's rows, else both     */
    int32_t radix_bits;    /* total partition bits of the hash join (0 = auto, <= 20)   */
    int32_t radix_bits1;   /* bits of the first partition pass (0 = auto)               */
    int32_t filter_bits;   /* log2 of the key-presence bitmap size (0 = auto, <= 30)    */
    int32_t heavy;         /* -1 auto, 0 off, 1 on, >= 2 on with this many rows making a key
                              frequent: frequent keys are joined as cross products          */
    int32_t theta_groups;  /* log2 of the theta/band group count (0 = auto, <= 10)      */
    int32_t nlj_tile_r;    /* R rows per nested-loop tile (0 = auto; multiple of 256)   */
    int32_t graphs;        /* 1: jn_batch captures and replays its phases as CUDA graphs */
    int32_t part_rows;     /* jn_batch: R rows per partition of an equi-join (0 = auto)  */
    int32_t host_io;       /* page-locked host buffers: bit 0 = the hash join reads its
                              input columns in place, bit 1 = emitted pairs are written in
                              place; otherwise copied (0 = copy both)                  */
    int32_t hash_path;     /* partitioning of the hash and sort-merge joins: 0 auto, 1 two
                              radix passes over both tables (pre-filter on both sides by
                              global presence bitmaps), 2 regions: one radix pass, then
                              one block per region splits it further and keeps the
                              pre-filter's bitmap slice of that region in shared memory,
                              thinning one table (the one `prefilter` names; the larger,
                              S on a tie, when both are named).  Auto = 2 unless the
                              columns are read in place from host memory or more than
                              18 partition bits are needed                              */
    int32_t table_rows;    /* R rows per shared-memory table of the hash and sort-merge
                              joins (the "bucket" a work item holds): 0 = the key type's
                              full table (4096 rows for int32 keys, 2048 for int64),
                              otherwise the full table when at least that size, else
                              half of it (jn_run_info.table_rows reports the size
                              used). jn_set_tuning accepts 0, 1024, 2048 and 4096     */
    int32_t sms;           /* SMs the context's persistent grids are sized for (0 = all;
                              more than the device has = all).  Fewer leaves room on
                              the device for another context's kernels              */
    int32_t reserved[3];
} jn_tuning;

/* Per-kernel launch statistics (profiling mode). */
typedef struct {
    char name[32];
    uint64_t launches;
    double ms;             /* summed device time between CUDA events around each launch */
} jn_kernel_stat;

/* What the last join on a context did (for benchmarks and tests). */
typedef struct {
    uint64_t result;            /* pairs produced (or counted)                      */
    uint64_t r_survivors;       /* R rows kept by the pre-filter (all when off)     */
    uint64_t s_survivors;
    uint64_t partitions;        /* partitions / groups / tiles of the join phase    */
    uint64_t work_items;        /* count/emit work items                            */
    uint64_t heavy_keys;        /* keys routed to the cross-product path            */
    uint64_t kernel_launches;   /* kernels launched by the call                     */
    int32_t prefilter;          /* tables the pre-filter thinned: 0 none, 1 both,
                                   2 only S, 3 only R                                */
    int32_t radix_bits;
    int32_t radix_bits1;
    int32_t filter_bits;
    uint64_t scratch_peak;      /* most scratch bytes the call held at once         */
    uint64_t heavy_pairs;       /* pairs emitted by the cross-product path          */
    uint64_t cartesian_bound;   /* what Eq. (rsize) would allocate for this run's
                                   decomposition: sum of |R_i| * |S_i| over the hash
                                   partitions (plus the frequent keys' exact cross
                                   products), over the theta join's compared and
                                   cross regions, or |R| * |S| for the nested loop;
                                   always >= result                                 */
    uint64_t hash_path;         /* partition path taken by the hash / sort-merge join:
                                   1 two radix passes, 2 regions (see jn_tuning)     */
    uint64_t table_rows;        /* R rows per shared-memory table the join used     */
    uint64_t reserved[1];
} jn_run_info;

typedef struct jn_ctx jn_ctx;

/* ------------------------------------------------------------ context --- */

/* Create a context on CUDA device `device` issuing work on `stream` (a
 * cudaStream_t; NULL = the legacy default stream).  Scratch and outputs are
 * stream-ordered allocations from the device's default memory pool (whose
 * release threshold the library raises so freed blocks are reused); outputs
 * may outlive the context. */
jn_status jn_create(jn_ctx** ctx, int device, void* stream);
void jn_destroy(jn_ctx* ctx);
jn_status jn_set_stream(jn_ctx* ctx, void* stream);
jn_status jn_set_tuning(jn_ctx* ctx, const jn_tuning* t);   /* NULL = defaults */
jn_status jn_get_tuning(const jn_ctx* ctx, jn_tuning* t);
const char* jn_status_str(jn_status s);
const char* jn_last_error(const jn_ctx* ctx);               /* text of the last failure */
const char* jn_version(void);

/* ------------------------------------------------------------ joins --- */

/* Exact result size of a join without writing pairs (the count pass that
 * replaces Eq. (rsize)'s estimate, Sec. 3.3.3).
 *   algo JN_ALGO_HASH : equality on key (pred must be NULL or op_a = JN_EQ
 *                       with no second conjunct);
 *   algo JN_ALGO_NLJ  : any jn_pred;
 *   algo JN_ALGO_THETA: pred->op_a on key, and, when pred->band >= 0, the band
 *                       on key2 (the jn_theta predicate).
 * *count (host) receives the number of pairs. */
jn_status jn_count(jn_ctx* ctx, int32_t algo, const jn_table* R, const jn_table* S,
                   const jn_pred* pred, uint64_t* count);

/* As jn_count, and also the separable checksum of the result multiset:
 *   checksum = sum over result pairs (r, s) of f(r) * g(s) mod 2^64,
 *   f(x) = mix(0x243F6A8885A308D3 ^ (uint32)x), g(x) = mix(0x13198A2E03707344 ^ (uint32)x),
 *   mix = the SplitMix64 output mixer.
 * This is the "results not stored" mode of Sec. 5.3 for outputs too large to
 * materialise.  checksum may be NULL. */
jn_status jn_aggregate(jn_ctx* ctx, int32_t algo, const jn_table* R, const jn_table* S,
                       const jn_pred* pred, uint64_t* count, uint64_t* checksum);

/* Output convention of the three joins:
 *   *out == NULL : the library allocates exactly *n_out pairs of device memory
 *                  (one allocation, after the count pass) and stores the
 *                  pointer in *out; release it with jn_free.  capacity is ignored.
 *   *out != NULL : a caller buffer of `capacity` pairs, device or host memory.
 *                  The kernels write 8-byte aligned device buffers (and, with
 *                  host_io bit 1, aligned page-locked host buffers) in place;
 *                  any other buffer is filled by a copy.
 *                  If the result has more pairs than capacity the call returns
 *                  JN_ERR_CAPACITY with *n_out = the required count and writes
 *                  nothing.  A host buffer is filled by a copy before return.
 * *n_out (host) receives the number of pairs written. */

/* Star join: the multi-table join Sec. 6 leaves to future work, as two of
 * this library's hash joins (a left-deep plan).  R carries two join columns,
 * key (fk1) and key2 (fk2); every row m of R, n1 of S1 and n2 of S2 with
 * R.key[m] == S1.key[n1] and R.key2[m] == S2.key[n2] gives one triple.
 *   - All key columns share one key type.  R's key2 and payload must be
 *     device memory (JN_ERR_INVALID otherwise); S1 and S2 may be host memory.
 *   - The first join's pair count must stay below 2^31 (JN_ERR_UNSUPPORTED).
 *   - Output: as the two-table joins (*out NULL: the library allocates the
 *     exact result, release it with jn_free_triples; otherwise a caller buffer
 *     of `capacity` triples in device or host memory, JN_ERR_CAPACITY with
 *     *n_out = the required count when it is too small). */
jn_status jn_star(jn_ctx* ctx, const jn_table* R, const jn_table* S1, const jn_table* S2, jn_triple** out,
                  uint64_t capacity, uint64_t* n_out);
jn_status jn_star_count(jn_ctx* ctx, const jn_table* R, const jn_table* S1, const jn_table* S2,
                        uint64_t* count);
void jn_free_triples(jn_ctx* ctx, jn_triple* p);

/* Nested-loop join (Sec. 3.3.1): every (R, S) pair is tested with `pred`
 * (NULL = equality on key).  Tiles of R are staged in shared memory and
 * compared against S rows held in registers. */
jn_status jn_nested_loop(jn_ctx* ctx, const jn_table* R, const jn_table* S, const jn_pred* pred,
                         jn_pair** out, uint64_t capacity, uint64_t* n_out);

/* Equi hash join (Sec. 3.3.2) with Algorithm 1's pre-filter (Sec. 3.1):
 * key-presence filters of both tables drop tuples whose key is absent from
 * the other table, a two-pass radix partition replaces the Map-Reduce
 * shuffle on key/alpha, and each partition is joined through a
 * shared-memory hash table built on its R rows. */
jn_status jn_hash(jn_ctx* ctx, const jn_table* R, const jn_table* S,
                  jn_pair** out, uint64_t capacity, uint64_t* n_out);

/* Equi sort-merge join: the third category of join algorithms in Sec. 2.3
 * (sort, then walk the tables in order), beside the nested-loop and hash
 * joins the paper builds.  The pre-filter, partitioning, frequent-key path,
 * count pass and exact allocation are those of jn_hash; within a partition
 * each chunk of R rows is sorted by key in shared memory and every S row
 * finds its run of equal keys by binary search.  Same arguments, result and
 * errors as jn_hash. */
jn_status jn_sort_merge(jn_ctx* ctx, const jn_table* R, const jn_table* S,
                        jn_pair** out, uint64_t capacity, uint64_t* n_out);

/* Theta join (Sec. 4.2, Algorithm 3).
 *   band < 0 : predicate R.key op S.key.  Both tables are cut into ranges with
 *              shared boundaries; off-diagonal regions whose ranges already
 *              decide the predicate are emitted as cross products without
 *              comparisons, diagonal regions are compared pair by pair, the
 *              rest are skipped.
 *   band >= 0: predicate (R.key op S.key) AND |R.key2 - S.key2| <= band.  The
 *              ranges are cut on key2; only region pairs within the band are
 *              compared.
 * Both tables need key2 when band >= 0. */
jn_status jn_theta(jn_ctx* ctx, const jn_table* R, const jn_table* S, int32_t op, int64_t band,
                   jn_pair** out, uint64_t capacity, uint64_t* n_out);

/* One join of a batch. */
typedef struct {
    jn_table R;
    jn_table S;
    int32_t op;        /* band < 0: must be JN_EQ (equi-join on key); band >= 0: op on key */
    int32_t reserved;  /* must be 0 */
    int64_t band;      /* < 0: equi-join; >= 0: band join |R.key2 - S.key2| <= band        */
} jn_join;

/* Runs `count` independent joins as one batch and writes all their pairs to
 * one device output (jn.h's output convention; the output must be device
 * memory, and *n_out receives the total).  first[i] and pairs[i] (host,
 * count words each) receive where join i's pairs start and how many there
 * are: they are out[first[i] .. first[i] + pairs[i]).  The equi-joins of a
 * batch share every phase (one radix pass over all their tables, one count
 * pass and one emit pass over a single work queue of (join, partition)
 * items), and so do its band joins (one range pass, one count pass and one
 * emit pass over (join, group) items).  Every join is counted before the
 * single exact output allocation; with tuning.graphs on, each phase is
 * replayed as a CUDA graph.  This is the batched form of the
 * Reducer = grid hierarchy of Sec. 3.3.4: many small joins fill the GPU
 * together instead of one launch sequence each. */
jn_status jn_batch(jn_ctx* ctx, int32_t count, const jn_join* joins, jn_pair** out, uint64_t capacity,
                   uint64_t* n_out, uint64_t* first, uint64_t* pairs);

/* Nested-loop join that allocates nothing, for callers that may not
 * allocate device memory: an application that owns every byte of the device
 * under a fixed memory plan, or a latency-critical loop that must not call
 * cudaMalloc / cudaFree (or any allocator, this library's pool included) and
 * the synchronisation they bring.  The paper has no counterpart; it is the
 * jn_nested_loop join without its allocations.
 *   - Scratch is one fixed device array inside the library (about 1 MiB per
 *     device, held until the process exits); a call handles at most 65536
 *     tiles of 1024 R rows by S_TILE S rows, i.e. ceil(|S| / S_TILE) *
 *     ceil(|R| / 1024) <= 65536 and ceil(|R| / 1024) <= 65535, where S_TILE
 *     is the nested loop's S tile (256 threads x JN_NLJ_SPT rows, 1024 with
 *     the default build).  Larger inputs return JN_ERR_INVALID.
 *   - Every call shares that array and it keeps the previous call's contents
 *     (the call rewrites what it reads): calls that overlap on the GPU, from
 *     any thread or stream, race and must be serialised by the caller.
 *   - Columns, output and `stream` must belong to the current device (the
 *     call uses that device's array); anything else returns JN_ERR_INVALID.
 *     The first call on a device looks up the array's device address.
 *   - Columns must be device memory; the output is a caller buffer of
 *     `capacity` pairs in device memory, 8-byte aligned (JN_ERR_INVALID
 *     otherwise).  When the result has more pairs,
 *     JN_ERR_CAPACITY is returned with *n_out = the required count and
 *     nothing is written.
 *   - Work is issued on `stream` (a cudaStream_t, NULL = legacy default).
 *     The call reads the count back into host memory and synchronises the
 *     stream, so it must not be issued on a stream that is being captured
 *     into a CUDA graph; the writes it then queues are complete when the
 *     stream reaches that point.
 * No context is used, so no error text is recorded: the status says it all. */
jn_status jn_nested_loop_noalloc(const jn_table* R, const jn_table* S, const jn_pred* pred, jn_pair* out,
                                 uint64_t capacity, uint64_t* n_out, void* stream);

/* Release an output allocated by a join (stream ordered on the context's
 * stream; with ctx == NULL, on the legacy default stream, so results may
 * outlive their context). */
void jn_free(jn_ctx* ctx, jn_pair* p);

/* Counts every join of a batch, as jn_batch would emit them, and writes no
 * pair: pairs[i] receives join i's result size, *total (may be NULL) their
 * sum.  Same arguments and checks as jn_batch; it runs the batch's shared
 * partition and count phases only, so a caller can size one output buffer
 * (or decide whether it fits) first. */
jn_status jn_batch_count(jn_ctx* ctx, int32_t count, const jn_join* joins, uint64_t* pairs, uint64_t* total);

/* Autotuner: times candidate tunings on these inputs -- the full join with a
 * library-allocated output that is freed at once, when the exact result fits
 * a quarter of the free device memory, else count and checksum -- applies the
 * fastest to the context and caches it per (algorithm, key type, size class);
 * *best (may be NULL) receives it.  The knobs tried never change a result: the hash and sort-merge joins'
 * partition bits and pre-filter, the theta join's group count, the nested
 * loop's R tile.  It stands in for the hand sweep of the partition parameter
 * alpha in Sec. 5.1.4 and 5.2.4. */
jn_status jn_autotune(jn_ctx* ctx, int32_t algo, const jn_table* R, const jn_table* S, const jn_pred* pred,
                      jn_tuning* best);
/* The same for a batch (rows per partition of its equi-joins, graphs on or
 * off), timing the batch's count phases. */
jn_status jn_autotune_batch(jn_ctx* ctx, int32_t count, const jn_join* joins, jn_tuning* best);

/* ------------------------------------------------------------- serving --- */

/* A request server over this library: requests are queued from any host
 * thread and run by `slots` worker threads, each with its own context and
 * CUDA stream, so the work of several requests overlaps on the device.
 * Small requests (|R| + |S| < coalesce_rows) waiting at the same time are
 * run together as one jn_batch (at most max_batch of them); larger requests
 * run alone after an exact count pass and wait until their scratch estimate
 * plus exact output fits memory_budget next to the outputs still held, as
 * long as another request is running (see jn_server_wait_any).
 * Tables registered with the server stay resident on the device.  The paper
 * has no serving layer; this is the request loop around its join method. */
typedef struct jn_server jn_server;

typedef struct {
    int32_t slots;           /* worker threads / streams, 1..16                     */
    int32_t coalesce_rows;   /* requests below this many rows are coalesced         */
    int32_t max_batch;       /* requests per coalesced batch, >= 1                  */
    int32_t graphs;          /* 1: batches replay their phases as CUDA graphs       */
    uint64_t memory_budget;  /* device bytes for scratch and held outputs           */
    int32_t small_slots;     /* of the slots, how many serve only requests below
                                coalesce_rows (a lane a small request never waits in
                                behind a large one); 0..slots-1                     */
    int32_t hold_wait_ms;    /* a request that does not fit next to the results the
                                client holds, while no other request runs, waits this
                                long (ms, >= 0) for a release, then is refused
                                (JN_ERR_OOM): bounded, so a client that releases in
                                submission order cannot deadlock the server          */
    int32_t small_sms;       /* with small_slots > 0: SMs the other workers' grids
                                leave free for the small-request lane
                                (jn_tuning.sms), >= 0                                */
    int32_t reserved;        /* must be 0                                           */
} jn_server_config;

typedef struct {
    int32_t r_handle;        /* > 0: registered table used as R; otherwise R below  */
    int32_t s_handle;        /* > 0: registered table used as S; otherwise S below  */
    jn_table R;              /* device tables, complete when submitted (the server reads
                                them on its own streams) and valid until completion  */
    jn_table S;
    int32_t op;              /* band < 0: JN_EQ; band >= 0: op on key               */
    int32_t reserved;        /* must be 0                                           */
    int64_t band;            /* < 0: equi-join; >= 0: band join on key2             */
} jn_request;

typedef struct {
    int32_t status;          /* jn_status of the request                            */
    int32_t reserved;
    uint64_t pairs;          /* result size                                         */
    jn_pair* out;            /* device pairs, owned by the server until released    */
    double queue_ms;         /* submit -> start on the device                       */
    double run_ms;           /* start -> pairs complete                              */
    double total_ms;         /* submit -> pairs complete                             */
} jn_result;

typedef struct {
    uint64_t submitted, completed, failed, batches, queued;
    uint64_t held_bytes, peak_bytes, resident_bytes;
    uint64_t kernel_launches;  /* kernels the workers launched (graph replays count their kernels) */
} jn_server_stats;

jn_status jn_server_create(jn_server** s, int device, const jn_server_config* cfg);
void jn_server_destroy(jn_server* s);          /* finishes queued requests, frees all */
/* Copies a table (host or device columns) into server-owned device memory. */
jn_status jn_server_register(jn_server* s, const jn_table* t, int32_t* handle);
jn_status jn_server_unregister(jn_server* s, int32_t handle);
jn_status jn_server_submit(jn_server* s, const jn_request* req, uint64_t* ticket);
jn_status jn_server_wait(jn_server* s, uint64_t ticket, jn_result* res);  /* blocks */
/* Returns the oldest completed request whose result no wait has returned yet
 * (its ticket and result): blocks up to timeout_ms (< 0: no limit), then
 * JN_ERR_TIMEOUT; JN_ERR_INVALID when every submitted request's result has
 * been returned.  Releasing results in completion order keeps held outputs
 * from filling the budget: a request that cannot fit next to held results
 * while no other request runs is refused with JN_ERR_OOM, not left waiting. */
jn_status jn_server_wait_any(jn_server* s, uint64_t* ticket, jn_result* res, int64_t timeout_ms);
jn_status jn_server_release(jn_server* s, uint64_t ticket);  /* frees the pairs of a done request */
jn_status jn_server_stats_get(jn_server* s, jn_server_stats* out);

/* ------------------------------------------------------- introspection --- */

/* Admission.  Every join finds its exact result size (the count pass) before
 * it allocates its output.  At that point a context
 *   - with a memory limit (bytes, 0 = none) refuses a run whose output plus
 *     the scratch it holds exceeds the limit: JN_ERR_OOM, nothing written,
 *     *n_out = the exact pair count;
 *   - with an admission hook calls it with the output bytes it is about to
 *     allocate (0 when the caller supplied device memory) and the scratch
 *     bytes it holds; any status but JN_OK stops the run with that status the
 *     same way.  The hook runs on the calling thread, between the count and
 *     the emit pass, and must not call into the same context.
 * This is how a caller admits work by exact bytes without a separate count
 * pass (jn_server uses it). */
typedef jn_status (*jn_admit_fn)(void* user, uint64_t out_bytes, uint64_t scratch_bytes);
jn_status jn_set_memory_limit(jn_ctx* ctx, uint64_t bytes);
jn_status jn_set_admission(jn_ctx* ctx, jn_admit_fn fn, void* user);  /* fn NULL: no hook */

jn_status jn_set_profiling(jn_ctx* ctx, int32_t on);  /* CUDA events around each launch */
/* Copies up to max entries (kernels with at least one launch) into out; *n =
 * entries written.  Synchronises the stream to resolve pending events. */
jn_status jn_kernel_stats(jn_ctx* ctx, jn_kernel_stat* out, int32_t max, int32_t* n);
jn_status jn_reset_stats(jn_ctx* ctx);
jn_status jn_last_run_info(const jn_ctx* ctx, jn_run_info* info);
uint64_t jn_launch_count(const jn_ctx* ctx);           /* kernels launched since creation */
int32_t jn_pointer_is_device(const void* p);            /* 1 if p is device (or managed) memory */

/* Diagnostic of the bounded device-side wait that every TMA staging pipeline
 * uses (not part of the join method).  One block on ctx's stream
 * initialises an mbarrier that expects one arrival and waits on its first
 * phase for at most `polls` polls (1 <= polls <= 2^20).  With arrive = 1 the
 * block arrives first and the wait completes: JN_OK.  With arrive = 0
 * nothing arrives, the wait runs out, the kernel records JN_ERR_TIMEOUT in
 * the context's device error word and returns, and the call returns
 * JN_ERR_TIMEOUT through the same read-back the joins use; the context
 * stays usable.  *elapsed_ns (may be NULL) receives the device time of the
 * wait.  Synchronises ctx's stream.  Errors: JN_ERR_INVALID (polls out of
 * range or no context), JN_ERR_CUDA. */
jn_status jn_selftest_wait(jn_ctx* ctx, uint32_t polls, int32_t arrive, uint64_t* elapsed_ns);

#ifdef __cplusplus
}
#endif

#endif /* JN_H */
