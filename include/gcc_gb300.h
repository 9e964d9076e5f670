/*
 * gcc_gb300.h -- C ABI of the GPU concurrency-control engine (sm_103a).
 *
 * The engine executes a batch of OLTP transactions concurrently on one GPU
 * under one of six concurrency-control schemes and returns, per transaction,
 * its commit status, its position in a commit order and the values it read.
 * It follows the paper's statement of the problem: transactions are run in
 * batches, one worker per transaction (Sec. III-C); read and write sets are
 * known before execution (Sec. IV-A, "Constraints"); an aborted transaction
 * restarts until it commits (Sec. IV-A, "Experimental Procedure"); every scheme
 * is serializable (Sec. III-E).  The committed transactions, executed serially
 * in the reported commit order from the same initial database, produce exactly
 * the reported reads and the final database.
 *
 * Conventions for every call:
 *  - Return value: GCC_OK or an error code; gcc_last_error() then gives a
 *    message (thread-local, valid until the next failing call on the thread).
 *  - Pointers are plain host or device pointers as stated per argument; no
 *    call takes ownership of caller memory.  Objects returned through `out`
 *    parameters are owned by the library until their destroy/free call.
 *  - Calls on one database must be ordered: issue them from one host thread
 *    and, for the asynchronous ones, on one stream (a NULL stream means the
 *    database's own stream).
 *  - Multi-byte fields are little-endian; structs below have no implicit
 *    padding.
 */
#ifndef GCC_GB300_H
#define GCC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gcc_status {
    GCC_OK = 0,
    GCC_ERR_INVALID = 1,   /* bad argument or malformed batch                   */
    GCC_ERR_CUDA = 2,      /* a CUDA runtime call failed                        */
    GCC_ERR_TIMEOUT = 3,   /* host wait ran out, or a device budget was spent   */
    GCC_ERR_NOMEM = 4,     /* device or host allocation failed                  */
    GCC_ERR_DEVICE = 5,    /* the kernel reported an error flag (see stats)     */
    GCC_ERR_CAPACITY = 6   /* batch larger than the database was created for,
                              or too many batches outstanding                   */
} gcc_status;

/* Batches submitted on one database and not yet released by gcc_batch_free. */
#define GCC_MAX_OUTSTANDING_BATCHES 256u

/* Concurrency-control schemes (Sec. II, Table I; Sec. III-E). */
typedef enum gcc_scheme {
    GCC_NO_WAIT_2PL = 0,   /* two-phase locking, abort when a lock is taken     */
    GCC_TO = 1,            /* basic timestamp ordering with a commit (dirty) bit */
    GCC_OCC = 2,           /* read-validate-write OCC with commit timestamps    */
    GCC_DET = 3,           /* deterministic conflict-ordered batch (GPUTx-like) */
    GCC_TICTOC = 4,        /* OCC with timestamps computed from per-record write
                              and read timestamps (TicToc, Table I) */
    GCC_2PL_WAIT_DIE = 5,  /* two-phase locking, an older transaction waits for a
                              younger exclusive holder, a younger one aborts */
    GCC_MVCC = 6           /* multi-version timestamp ordering: writes make new
                              versions, a read takes the newest version older
                              than its timestamp (Sec. II, Table I; Sec. III-E);
                              key-value databases */
} gcc_scheme;

typedef enum gcc_schema {
    GCC_SCHEMA_KV = 0,           /* one table of n_records x n_fields slots      */
    GCC_SCHEMA_ORDER_ENTRY = 1   /* TPC-C-shaped warehouse/district/customer/... */
} gcc_schema;

/* Op kinds.  Key-value: READ returns the slot; ADD returns the old slot and
 * adds the operand (8-byte slots: modulo 2^64; 16-byte slots: lo modulo 2^64
 * and bytes 8-9 as a u16 modulo 2^16, bytes 10-15 unchanged).
 * Order-entry kinds implement the NewOrder and Payment procedures, one op per
 * record access, in this fixed layout (row numbering as in the table ids
 * below; reads are (lo, hi) pairs):
 *   NewOrder: W_READ(w) -> (w_tax, 0); D_NEWORDER(district) -> (d_next_o_id,
 *     d_tax), next_o_id += 1; C_READ(customer) -> (c_discount, c_balance);
 *     then per line: I_READ(item) -> (i_price, 0), S_NEWORDER(stock row,
 *     operand qty, remote) -> (s_quantity, s_order_cnt) with s_quantity -= qty
 *     (+91 when the old quantity was below qty + 10), s_ytd += qty,
 *     s_order_cnt += 1, s_remote_cnt += remote.  At commit the order
 *     (o_id = the d_next_o_id read), its new-order flag and its lines
 *     (amount = qty * i_price) are inserted.
 *   Payment: W_PAY(w, h) -> (w_ytd, 0); D_PAY(district, h) -> (d_ytd, 0);
 *     C_PAY(customer, h) -> (c_balance, c_payment_cnt), c_balance -= h,
 *     c_ytd_payment += h, c_payment_cnt += 1; or, naming the customer by last
 *     name, C_PAY_BY_NAME(key = the customer's district, aux = last-name id,
 *     h): among the district's customers with that c_last, ordered by c_first
 *     and then by customer number, the one at position ceil(n/2) is paid as
 *     by C_PAY (a name nobody in the district has makes the transaction
 *     invalid).  The paper's payment names its customer (Sec. IV-A); the
 *     selection rule is this library's reading.  The lookup uses a
 *     per-district index sorted by (last, first, number) and binary search
 *     (the sorted-array index of Sec. III-D), built whenever table 22 or 23
 *     is loaded, and happens before the transaction touches any control word
 *     (names are never written). */
enum gcc_op_kind {
    GCC_OP_READ = 0,
    GCC_OP_ADD = 1,
    GCC_OE_W_READ = 16,
    GCC_OE_W_PAY = 17,
    GCC_OE_D_NEWORDER = 18,
    GCC_OE_D_PAY = 19,
    GCC_OE_C_READ = 20,
    GCC_OE_C_PAY = 21,
    GCC_OE_I_READ = 22,
    GCC_OE_S_NEWORDER = 23,
    GCC_OE_C_PAY_BY_NAME = 24
};

enum gcc_txn_type { GCC_TXN_KV = 0, GCC_TXN_NEW_ORDER = 1, GCC_TXN_PAYMENT = 2 };

/* Per-transaction outcome. */
enum gcc_txn_status {
    GCC_TXN_PENDING = 0,     /* not executed (the batch was cut short)           */
    GCC_TXN_COMMITTED = 1,
    GCC_TXN_TIMEOUT = 2,     /* attempt budget, wait budget or deadline spent     */
    GCC_TXN_INVALID = 3      /* bad key/field/kind, duplicate key, too many ops  */
};

/* A transaction: ops[first_op .. first_op + n_ops).  Transactions are given in
 * transaction-id order (index = id); their op ranges must not overlap and must
 * increase with the id.  GCC_DET orders conflicting accesses by op position,
 * so there the ranges must tile ops[0 .. n_ops) exactly, in id order; an op
 * outside every range makes later accesses to its record wait until
 * wait_budget_ns runs out (GCC_TXN_TIMEOUT). */
typedef struct gcc_txn {
    uint32_t first_op;
    uint16_t n_ops;
    uint16_t type;           /* gcc_txn_type */
} gcc_txn;

/* An op descriptor.  key: record number (key-value) or row (order-entry);
 * field: key-value field index; kind: gcc_op_kind.  Keys within one
 * transaction must be distinct (record-granularity conflicts). */
typedef struct gcc_op {
    uint32_t key;
    uint8_t field;
    uint8_t kind;
    uint16_t aux;            /* C_PAY_BY_NAME: last-name id; otherwise 0 */
} gcc_op;

/* An op operand or a value read: two 64-bit lanes. */
typedef struct gcc_operand {
    uint64_t lo;
    uint64_t hi;
} gcc_operand;

typedef struct gcc_txn_result {
    uint32_t status;         /* gcc_txn_status */
    uint32_t attempts;       /* executions started, including the committing one */
    uint64_t commit_order;   /* committed: 0..n_committed-1, a serial order;
                                otherwise UINT64_MAX */
} gcc_txn_result;

typedef struct gcc_db_desc {
    uint32_t schema;           /* gcc_schema */
    uint32_t field_bytes;      /* key-value: 8 or 16 */
    uint64_t n_records;        /* key-value: records (<= 2^31) */
    uint32_t n_fields;         /* key-value: fields per record (1..255) */
    uint32_t n_warehouses;     /* order-entry: W (1..1024) */
    uint32_t order_cap;        /* order-entry: order slots per district (>= 3000) */
    uint32_t max_ops_per_txn;  /* upper bound on gcc_txn.n_ops (1..64) */
    uint64_t max_batch_txns;   /* upper bound on transactions per batch */
    uint64_t max_batch_ops;    /* upper bound on ops per batch (< 2^32) */
    int32_t device;            /* CUDA device ordinal */
    uint32_t reserved;         /* 0 */
} gcc_db_desc;

/* Launch and retry policy.  Zero fields take the defaults in brackets. */
typedef struct gcc_exec_params {
    uint32_t lanes_per_txn;    /* lanes of a warp that cooperate on one
                                  transaction: 1,2,4,8,16,32 [16] */
    uint32_t warps_per_block;  /* 1..32 [8] */
    uint32_t blocks_per_sm;    /* resident blocks per SM [occupancy limit] */
    uint32_t collapse;         /* 1 = collapse same-key lock attempts inside a
                                  warp before they reach global atomics [1];
                                  2 = off */
    uint32_t backoff_base_ns;  /* first retry delay, doubled per abort, with
                                  random jitter [128] */
    uint32_t backoff_cap_ns;   /* largest retry delay [1000000] */
    uint32_t max_attempts;     /* per transaction, then GCC_TXN_TIMEOUT [2^24] */
    uint32_t read_retries;     /* re-reads of a record seen mid-update before
                                  the attempt aborts [8] */
    uint64_t wait_budget_ns;   /* deterministic scheme: bound on one wait [2 s] */
    uint64_t deadline_ns;      /* whole-kernel budget, then remaining work ends
                                  as GCC_TXN_TIMEOUT [60 s] */
    uint64_t seed;             /* retry jitter and abort injection */
    uint32_t inject_abort_ppm; /* test hook: abort an attempt at its commit point
                                  with this probability per million [0] */
    uint32_t immediate_restart;/* 1 = restart an aborted transaction at once, with
                                  no delay (the paper's policy) [0] */
    uint32_t det_dataflow;     /* GCC_DET: 0 = evaluate each record's chain in one
                                  pass over the batch's accesses sorted by record
                                  (key-value: prefix sums; order-entry: one warp
                                  per record applies its ops in id order)
                                  [default; key-value needs n_records *
                                  n_fields below 2^32, else the batch is
                                  refused with GCC_ERR_CAPACITY]; 1 = run op
                                  by op in the execute
                                  kernel, each op waiting for its predecessors
                                  (a read for the earlier writes, a write for
                                  every earlier access); 2 = the same with every
                                  access waiting for every earlier access to
                                  its record, reads included (GaccO-style
                                  hand-off, Sec. II-C) */
    uint32_t retry_queue;      /* 2PL/TO/OCC: 1 = an aborted transaction that
                                  conflicted on a record waits, holding nothing,
                                  in a FIFO queue for that record and re-attempts
                                  when served [1]; 2 = off (randomized backoff
                                  after every abort) */
    uint32_t queue_turn_ns;    /* estimated time per queue turn: a waiter n
                                  turns from its own sleeps about n - 1 turns
                                  before looking again [1000] */
    uint32_t queue_width;      /* transactions a retry queue lets attempt at
                                  once [1] */
    uint32_t queue_after;      /* aborts of a transaction before it uses retry
                                  queues; 1 = from its first abort [2PL, TO:
                                  16; OCC: 64 -- an OCC abort nearly always
                                  means another transaction committed, so its
                                  retries rarely need queueing] */
    uint32_t group_commit;     /* OCC on key-value databases: transactions per
                                  commit unit, 2..8 (1 = off) [1].  The
                                  batch's transactions are keyed by their
                                  most-written record; a key's transactions
                                  (in id order) form units that one lane group
                                  attempts together: one lock per distinct
                                  written record, consecutive commit
                                  timestamps, per-member validation, writes
                                  composed in timestamp order; members that
                                  fail retry.  At most 255 ops per unit: the
                                  unit size is cut to 255 / max_ops_per_txn */
    uint32_t group_min_writes; /* writes in the batch that make a record a key
                                  of units [32] */
    uint32_t reserved;         /* 0 */
} gcc_exec_params;

typedef struct gcc_batch_stats {
    uint64_t n_txns;
    uint64_t committed;
    uint64_t aborts;           /* aborted attempts (abort rate = aborts/committed) */
    uint64_t timeouts;
    uint64_t invalid;
    uint64_t max_attempts;     /* largest attempts count of any transaction */
    uint32_t device_error;     /* GCC_DEVERR_* bits */
    uint32_t scheme;
    double elapsed_ms;         /* device time of the batch (submit/wait only) */
    double prep_ms;            /* stage times from CUDA events on the batch's
                                  stream: control-word reset, batch begin and
                                  deterministic preprocessing */
    double kernel_ms;          /* the execute kernel */
    double order_ms;           /* dense commit ranks */
    uint32_t kernel_launches;  /* kernels this execution launched */
    uint32_t grid_blocks;      /* blocks of the execute kernel */
    uint64_t atomics;          /* global atomic read-modify-write operations the
                                  execute kernel issued (lock and version CASes,
                                  timestamp and fetch tickets, counters, queue
                                  tickets; 0 for the deterministic passes that
                                  run without it) */
} gcc_batch_stats;

/* Stage times of one past execution (see gcc_stage_history). */
typedef struct gcc_stage_times {
    double prep_ms;
    double kernel_ms;
    double order_ms;
    uint32_t scheme;
    uint32_t n_txns;
    uint32_t kernel_launches;
    uint32_t grid_blocks;
} gcc_stage_times;

/* device_error bits */
#define GCC_DEVERR_WAIT_BUDGET   0x1u   /* a deterministic wait ran out        */
#define GCC_DEVERR_DEADLINE      0x2u   /* deadline_ns passed                  */
#define GCC_DEVERR_TS_OVERFLOW   0x4u   /* OCC/TO: the batch used 2^32-1 or
                                           more timestamps; its commit order
                                           is not valid                       */
#define GCC_DEVERR_ATTEMPTS      0x8u   /* a transaction hit max_attempts      */
#define GCC_DEVERR_INVALID       0x10u  /* a transaction was malformed         */
#define GCC_DEVERR_INSERT        0x20u  /* an order insert had no free slot    */

typedef struct gcc_db gcc_db;
typedef struct gcc_batch gcc_batch;

/* Create a database on desc->device: allocates its tables (zeroed), the
 * per-record concurrency-control words and the scratch needed for batches
 * up to the stated maxima.  Paper: tables on the GPU are fixed-size arrays
 * whose size does not change during execution (Sec. III-D, "DBMS Building
 * Blocks"), and all table data is resident in device memory before any
 * transaction runs (Sec. IV-A, "Constraints"); one concurrency-control word
 * per record, as in Table II (Sec. III-E).  Key-value: one table (id 0).  Order-entry: one
 * table per column (ids 0..21 in this order: w_ytd, w_tax, d_ytd, d_tax,
 * d_next_o_id, c_balance, c_ytd_payment, c_payment_cnt, c_discount, i_price,
 * s_quantity, s_ytd, s_order_cnt, s_remote_cnt, o_c_id, o_ol_cnt,
 * o_all_local, no_flag, ol_i_id, ol_supply_w_id, ol_quantity, ol_amount,
 * c_last, c_first; all int64; order slot = district * order_cap + o_id - 1,
 * line = slot * 15 + l; c_last and c_first are the customers' name keys,
 * read only by payments by last name).
 * Errors: GCC_ERR_INVALID (desc out of range), GCC_ERR_NOMEM, GCC_ERR_CUDA. */
gcc_status gcc_db_create(const gcc_db_desc *desc, gcc_db **out);

/* Free every device allocation of db (synchronises its stream).  NULL is a
 * no-op. */
gcc_status gcc_db_destroy(gcc_db *db);

/* Number of tables and the byte size of one table (0 for a bad id). */
uint32_t gcc_table_count(const gcc_db *db);
uint64_t gcc_table_bytes(const gcc_db *db, uint32_t table_id);

/* Copy nbytes (must equal gcc_table_bytes) into table table_id from a host
 * (src_on_device = 0) or device pointer, and reset the concurrency-control
 * words.  Synchronous.  Paper: the host generates the tables and transfers
 * them to GPU memory before execution (Sec. IV-A, "Experimental Procedure";
 * the CPU side coordinates data generation and initialisation, Sec. III-C).
 * Errors: GCC_ERR_INVALID (NULL db or src, bad table id, nbytes differs from
 * the table's size), GCC_ERR_CUDA.  src stays owned by the caller.  Key-value layout: field-major, slot (key, field) at
 * byte (field * n_records + key) * field_bytes. */
gcc_status gcc_load_table(gcc_db *db, uint32_t table_id, const void *src,
                          uint64_t nbytes, int src_on_device);

/* Fill key-value table 0 on the device with seeded initial values and reset
 * the concurrency-control words, as gcc_load_table does (synchronous).  Slot
 * (key, field) takes output number key * n_fields + field + 1 of splitmix64
 * seeded with `seed` (the YCSB-shaped table of Sec. IV-A, generated where it
 * lives instead of copied in); a 16-byte slot holds that output in bytes 0-7,
 * the low 16 bits of the same output number under the seed splitmix64(seed, 2)
 * in bytes 8-9, and zeros in bytes 10-15.  Errors: GCC_ERR_INVALID (NULL db,
 * an order-entry database, table_id != 0), GCC_ERR_CUDA. */
gcc_status gcc_init_table_seeded(gcc_db *db, uint32_t table_id, uint64_t seed);

/* Copy table table_id out (synchronous; waits for prior work on the stream)
 * to a host (dst_on_device = 0) or device pointer of nbytes (must equal
 * gcc_table_bytes).  Paper: updates stay in device memory during execution
 * (Sec. IV-A, "Constraints") and correctness is checked on the host after
 * execution (Sec. III-D, "Measurements and Verification"); this is the
 * snapshot such a check compares.  Errors: GCC_ERR_INVALID (NULL pointer,
 * bad table id, wrong nbytes), GCC_ERR_CUDA.  dst stays owned by the
 * caller. */
gcc_status gcc_db_read_table(gcc_db *db, uint32_t table_id, void *dst,
                             uint64_t nbytes, int dst_on_device);

/* Fill *p with the defaults. */
gcc_status gcc_default_params(gcc_exec_params *p);

/* Submit a batch asynchronously.  Paper: transactions run in batches with
 * one worker per transaction (Sec. III-C, batch execution model); every
 * transaction's reads and writes are known before execution, given here as
 * its op list (Sec. IV-A, "Constraints"); a transaction that fails on a
 * conflict restarts until it commits (Sec. IV-A, "Experimental Procedure");
 * every scheme gives serializable results (Sec. III-E).
 * txns/ops/operands are host pointers
 * (copied before the call returns) or, with inputs_on_device = 1, device
 * pointers that must stay valid until gcc_batch_wait returns.  params may be
 * NULL (defaults).  stream: a cudaStream_t, or NULL for the database's own
 * stream.  Errors: GCC_ERR_INVALID (n_ops/op ranges inconsistent, bad
 * scheme), GCC_ERR_CAPACITY (beyond the create-time maxima, or
 * GCC_MAX_OUTSTANDING_BATCHES batches not yet freed), GCC_ERR_NOMEM,
 * GCC_ERR_CUDA.  Per-transaction problems (bad keys, duplicates) are not
 * errors here: those transactions come back as GCC_TXN_INVALID. */
gcc_status gcc_txn_batch_submit(gcc_db *db, gcc_scheme scheme, const gcc_txn *txns,
                                uint32_t n_txns, const gcc_op *ops,
                                const gcc_operand *operands, uint64_t n_ops,
                                int inputs_on_device, const gcc_exec_params *params,
                                void *stream, gcc_batch **out);

/* Wait up to timeout_ns (UINT64_MAX = forever) for the batch, then copy its
 * per-transaction results (n_txns entries) and read values (n_ops entries,
 * indexed like ops) to host (outputs_on_device = 0) or device pointers; any
 * output pointer may be NULL.  Paper: the batch is timed from the
 * initialisation of the scheme to the completion of every transaction, and
 * the abort rate is aborts per committed transaction (Sec. IV-A, "Metric
 * Selection"); stats carries both, and per-stage times (Sec. III-D,
 * "Measurements and Verification").  The outputs stay owned by the caller.  GCC_ERR_TIMEOUT leaves the batch waitable
 * again.  GCC_ERR_DEVICE when stats.device_error is nonzero (outputs are
 * still written). */
gcc_status gcc_batch_wait(gcc_batch *batch, uint64_t timeout_ns, gcc_txn_result *results,
                          gcc_operand *read_values, gcc_batch_stats *stats,
                          int outputs_on_device);

/* Release a batch (waits for it first).  NULL is a no-op. */
gcc_status gcc_batch_free(gcc_batch *batch);

/* Device-resident form of submit: every pointer is a device pointer, the
 * results are written to d_results (n_txns) and d_reads (n_ops), and the
 * call only enqueues work on `stream` (NULL = the database's stream).  No
 * allocation happens here.  Statistics of the latest execution are read
 * with gcc_last_stats. */
gcc_status gcc_execute(gcc_db *db, gcc_scheme scheme, const gcc_txn *d_txns,
                       uint32_t n_txns, const gcc_op *d_ops,
                       const gcc_operand *d_operands, uint64_t n_ops,
                       const gcc_exec_params *params, gcc_txn_result *d_results,
                       gcc_operand *d_reads, void *stream);

/* Statistics of the latest gcc_execute / submit on db (synchronises its
 * stream; elapsed_ms is 0 for gcc_execute). */
gcc_status gcc_last_stats(gcc_db *db, gcc_batch_stats *stats);

/* Stage times of the latest executions on db, oldest first: up to max_entries
 * of the last 256, written to out; *n_out receives the count.  Synchronises
 * the streams they ran on. */
gcc_status gcc_stage_history(gcc_db *db, uint32_t max_entries, gcc_stage_times *out,
                             uint32_t *n_out);

/* Batched form: many independent key-value batches, each on its own
 * database, executed by one persistent-kernel launch (Sec. IV-C studies the
 * effect of launch parameters; here the launch is shared).  All databases
 * share one device and slot width; each appears at most once.  Device
 * pointers, as for gcc_execute. */
typedef struct gcc_multi_batch {
    gcc_db *db;
    const gcc_txn *d_txns;
    uint32_t n_txns;
    uint32_t reserved;         /* 0 */
    const gcc_op *d_ops;
    const gcc_operand *d_operands;
    uint64_t n_ops;
    gcc_txn_result *d_results;
    gcc_operand *d_reads;
} gcc_multi_batch;

typedef struct gcc_multi_plan gcc_multi_plan;

/* Build a launch plan for `n` batches (at most 256) under any scheme:
 * uploads the batch descriptors, allocates the plan's scratch (sort
 * buffers for all transactions) and puts every database's control words in a
 * state the scheme can start from.  Under GCC_DET every batch runs its
 * database's own prefix-sum evaluation (as gcc_execute's default
 * deterministic path; n_records * n_fields below 2^32, else
 * GCC_ERR_CAPACITY), the batches spread over up to eight side streams forked
 * from and joined into the launch stream, so that their pipelines overlap.
 * The batch arrays must stay valid while the plan is used.  Synchronous. */
gcc_status gcc_multi_plan_create(gcc_scheme scheme, const gcc_multi_batch *batches, uint32_t n,
                                 const gcc_exec_params *params, gcc_multi_plan **out);

/* Enqueue one execution of every batch of the plan on `stream` (NULL = the
 * plan's stream): batch states reset, one persistent kernel over all
 * transactions (OCC, TO and the two 2PL schemes, TicToc, MVCC; MVCC then
 * writes every database's newest versions into its table), commit ranks
 * (OCC and TO by the plan's shared clock, TicToc by (timestamp, sequence
 * number), MVCC by each batch's own timestamps, both 2PL schemes by each
 * database's lock-point counter).  With use_graph != 0 the sequence is captured
 * once into a CUDA graph (on the plan's stream) and replayed.  Allocates
 * nothing.  Between launches, run no other scheme on the plan's databases
 * (GCC_ERR_INVALID otherwise). */
gcc_status gcc_multi_launch(gcc_multi_plan *plan, int use_graph, void *stream);

/* Statistics of batch i of the latest launch (synchronises the device). */
gcc_status gcc_multi_stats(gcc_multi_plan *plan, uint32_t i, gcc_batch_stats *stats);

/* Free the plan (waits for its stream).  NULL is a no-op. */
gcc_status gcc_multi_plan_destroy(gcc_multi_plan *plan);

/* Served form: a request loop that forms batches continuously.  Each lane
 * serves one database: arriving transactions join the lane's forming batch
 * until its transaction cap or its write-set budget (16 bytes per writing op)
 * is reached, until its oldest request has waited max_delay_ns, or, sooner,
 * as soon as none of the lane's batches is in flight (waiting gains nothing
 * while the lane's device work is idle; under load batches grow up to the
 * delay or the caps); the batch is then copied to the device, executed and
 * copied back on the lane's own
 * streams while the next batch forms.  Up to `depth` batches per lane are in
 * flight; lanes run concurrently.  Batches of one lane execute in formation
 * order (batch_seq), so a lane's committed requests, in (batch_seq,
 * commit_order) order, form one serial history of its database. */
typedef struct gcc_server_lane {
    gcc_db *db;
    uint32_t scheme;             /* gcc_scheme */
    uint32_t max_batch_txns;     /* <= the database's max_batch_txns */
    uint64_t write_budget_bytes; /* per batch [16 * max_batch_txns * 16] */
    uint64_t max_delay_ns;       /* [200000] */
    uint32_t depth;              /* batches in flight, 1..8 [3] */
    uint32_t reserved;           /* 0 */
} gcc_server_lane;

typedef struct gcc_completion {
    uint64_t request;            /* id from gcc_server_enqueue / trace index */
    uint32_t lane;
    uint32_t status;             /* gcc_txn_status */
    uint64_t batch_seq;          /* per lane, in execution order */
    uint64_t commit_order;       /* within the batch */
    uint64_t arrival_ns;         /* host steady clock */
    uint64_t done_ns;            /* when the server saw the result on the host */
} gcc_completion;

typedef struct gcc_server gcc_server;

/* Create a server over n_lanes lanes (distinct databases, one device).
 * Allocates every slot's pinned host and device buffers up front. */
gcc_status gcc_server_create(const gcc_server_lane *lanes, uint32_t n_lanes,
                             const gcc_exec_params *params, gcc_server **out);

/* Admit one transaction (host memory, copied) to `lane`.  Its ops start at
 * ops[0] (txn->first_op is ignored).  arrival_ns is its arrival time on the
 * host steady clock (see gcc_server_now_ns).  *request_id receives its id.
 * GCC_ERR_CAPACITY when txn->n_ops exceeds the database's max_ops_per_txn or
 * the lane's batch op capacity (min(max_batch_txns * max_ops_per_txn,
 * max_batch_ops)). */
gcc_status gcc_server_enqueue(gcc_server *s, uint32_t lane, const gcc_txn *txn,
                              const gcc_op *ops, const gcc_operand *operands,
                              uint64_t arrival_ns, uint64_t *request_id);

/* Launch batches that are full or past their delay, collect finished ones. */
gcc_status gcc_server_pump(gcc_server *s);

/* Launch every forming batch and wait for all of them. */
gcc_status gcc_server_drain(gcc_server *s);

/* Pop up to max completions (oldest first); read values of each completed
 * request go to reads_out consecutively (may be NULL). */
gcc_status gcc_server_completions(gcc_server *s, gcc_completion *out, gcc_operand *reads_out,
                                  uint64_t reads_capacity, uint32_t max, uint32_t *n_out);

/* Open-loop replay of a request trace: request i (ops at
 * ops[txns[i].first_op ..]) arrives at start + arrival_offset_ns[i] for lane
 * lane_of[i]; the loop admits arrivals, launches and collects batches until
 * every request has completed.  Each lane runs on two host threads of its
 * own, one admitting arrivals and launching batches, one collecting finished
 * batches; the call returns when every lane is done.  A lane admits its requests in index
 * order, so arrival_offset_ns should be nondecreasing.  out[i] and
 * reads_out[txns[i].first_op ..] receive the outcome of request i.  An error
 * in a lane stops that lane; the call returns the lowest failing lane's
 * status, its message prefixed by the lane.
 * GCC_ERR_INVALID (nothing run) for a bad lane or a request too large for its
 * lane, as in gcc_server_enqueue. */
gcc_status gcc_server_run_trace(gcc_server *s, uint32_t n, const uint32_t *lane_of,
                                const gcc_txn *txns, const gcc_op *ops,
                                const gcc_operand *operands, const uint64_t *arrival_offset_ns,
                                gcc_completion *out, gcc_operand *reads_out);

/* Host steady clock in nanoseconds (the clock of arrival_ns / done_ns). */
uint64_t gcc_server_now_ns(void);

/* Totals of a lane since creation: committed transactions, aborted
 * attempts and batches completed. */
gcc_status gcc_server_lane_totals(gcc_server *s, uint32_t lane, uint64_t *committed,
                                  uint64_t *aborts, uint64_t *batches);

/* Drain and free the server.  NULL is a no-op. */
gcc_status gcc_server_destroy(gcc_server *s);

/* Launch-parameter search space for gcc_autotune.  The paper finds that the
 * number of active lanes per warp and warps per block move throughput by up
 * to 10x (Sec. IV-C, Exp-3 to Exp-5); this searches the engine's equivalents
 * plus the retry-delay cap.  Zero counts take the defaults in brackets. */
typedef struct gcc_tune_space {
    uint32_t n_lanes;          /* [5]: lanes_per_txn in {2, 4, 8, 16, 32} */
    uint32_t lanes[6];
    uint32_t n_warps;          /* [4]: warps_per_block in {4, 8, 16, 32} */
    uint32_t warps[8];
    uint32_t n_caps;           /* [3]: backoff_cap_ns in {65536, 1000000, 16000000} */
    uint32_t caps[4];
    uint32_t steps;            /* timed executions per point [2] */
    uint32_t warmup;           /* untimed executions per point [1] */
    uint64_t point_deadline_ns;/* kernel deadline per execution [5 s] */
} gcc_tune_space;

typedef struct gcc_tune_report {
    uint32_t points;           /* points measured (shapes that fit an SM) */
    uint32_t best_index;       /* in measurement order */
    double best_txn_per_s;     /* committed transactions per second at the best */
    double default_txn_per_s;  /* the same with gcc_default_params */
} gcc_tune_report;

/* Grid search for the launch parameters that commit the given batch fastest:
 * every point of `space` runs `warmup` + `steps` executions of the batch
 * (device pointers, as gcc_execute) on `stream`, timed with CUDA events;
 * *best receives the winning parameters.  The batch executes many times, so
 * the database's contents change; tune on a copy when that matters.
 * Synchronous. */
gcc_status gcc_autotune(gcc_db *db, gcc_scheme scheme, const gcc_txn *d_txns, uint32_t n_txns,
                        const gcc_op *d_ops, const gcc_operand *d_operands, uint64_t n_ops,
                        gcc_txn_result *d_results, gcc_operand *d_reads,
                        const gcc_tune_space *space, gcc_exec_params *best,
                        gcc_tune_report *report, void *stream);

/* Deterministic (GCC_DET) execution of one key-value batch that allocates
 * nothing.  The paper has no counterpart to this call; it exists for callers
 * that cannot allocate device memory -- for instance a host application whose
 * device memory is reserved up front by another framework's caching
 * allocator, or a latency-critical loop where cudaMalloc's implicit device
 * synchronisation is unacceptable.  The caller passes device pointers to the
 * table (field-major slots as in gcc_load_table, updated in place), the batch
 * and the outputs; the result equals gcc_execute with GCC_DET on a database
 * holding the same table.  All scratch lives in one static device array of
 * about 1.8 MB, which every GPU that loads this library keeps until the
 * process exits.  Limits: n_records, n_ops and n_txns at most 65536 each
 * (GCC_ERR_CAPACITY beyond), max_ops_per_txn in 1..64.  The first call on a
 * device looks up the array's device address; make that first call before
 * any stream capture.  Every call reuses the same array, so calls that
 * overlap on the GPU (other streams, other host threads) race with each
 * other.  The call only enqueues work on `stream` (NULL = legacy default
 * stream); per-transaction outcomes land in d_results.  Batch-level counters
 * and device error bits (gcc_batch_stats) stay in the static array and are
 * not reported: a caller learns of a malformed transaction or a spent wait
 * budget only from the status of each entry of d_results, so check them all.
 * Errors: GCC_ERR_CAPACITY (a size above its limit), GCC_ERR_INVALID (bad
 * slot width, field count, op bound or NULL pointer, or a launch shape that
 * does not fit an SM), GCC_ERR_CUDA. */
gcc_status gcc_det_execute_noalloc(void *d_table, uint32_t n_records, uint32_t n_fields,
                                   uint32_t field_bytes, const gcc_txn *d_txns, uint32_t n_txns,
                                   const gcc_op *d_ops, const gcc_operand *d_operands,
                                   uint32_t n_ops, uint32_t max_ops_per_txn,
                                   gcc_txn_result *d_results, gcc_operand *d_reads,
                                   void *stream);

/* Memory-system figures of one GPU, measured with the PTX operations the
 * schemes use.  They are the denominators of the execute kernels' rooflines:
 * bandwidth (random sectors, atomics on distinct words) when records are
 * spread, and the latency of one contended record when hot records serialise
 * their writers (Sec. IV-C finds contention decisive: every serializable
 * read-modify-write chain on one record pays its protocol's round trips once
 * per link).  The paper has no such call. */
typedef struct gcc_memory_probe {
    double hbm_load_ns;        /* dependent relaxed loads of lines not in L2 */
    double l2_load_ns;         /* dependent relaxed loads of L2-resident lines */
    double l2_load_acquire_ns; /* the same with acquire loads */
    double l2_atomic_ns;       /* dependent atomicAdd(0) on L2-resident words */
    double l2_cas_ns;          /* dependent (failing) 64-bit CAS on L2-resident words */
    double gather32_gbs;       /* random 32-byte sectors of a 1 GiB buffer, all SMs,
                                  GB/s: the best of gather32_by_inflight_gbs */
    double cas_distinct_gops;  /* successful 64-bit CAS, one word per 32 B sector and
                                  thread, all SMs, 1e9 per second */
    double add_same_gops;      /* atomicAdd on one word, one lane per warp, all SMs */
    double lock_handoff_ns;    /* one lock word: test, CAS acquire, release
                                  store; ns per acquisition, best over 2, 16,
                                  sm_count and `contenders` contending warps */
    double occ_cycle_ns;       /* one record under the OCC commit sequence (acquire
                                  version, read value, CAS lock, fence, ticket, write,
                                  fence, publish); ns per commit, best over the
                                  same contender counts */
    double occ_cycle_busy_ns;  /* the same with `contenders` warps */
    uint32_t sm_count;
    uint32_t contenders;       /* 8 warps per SM (one lane each) */
    uint32_t lock_best_contenders;  /* contending warps at lock_handoff_ns */
    uint32_t occ_best_contenders;   /* contending warps at occ_cycle_ns */
    double fence_ns;           /* fence.acq_rel.gpu with no memory operation in
                                  flight, one thread (least over the placements
                                  of occ_link_ns) */
    double atomic_acq_rel_ns;  /* dependent acquire-release atomicAdd, one word
                                  (least over the same placements) */
    double occ_link_ns;        /* one uncontended link of the OCC commit chain as
                                  the execute kernel runs it (acquire version,
                                  CAS lock, acquire-release commit timestamp,
                                  one validation load, value store, release
                                  publish): the least time per committed
                                  writer of one record, least over eight
                                  placements of the thread (the SMs of both
                                  dies) */
    double occ_link_max_ns;    /* the greatest over the same placements */
    double gather32_by_inflight_gbs[3]; /* random 32-byte sectors with 4, 8 and
                                  16 sectors in flight per thread */
    uint32_t gather32_best_inflight;    /* in-flight count of gather32_gbs */
    uint32_t reserved;
} gcc_memory_probe;

/* Run the probes on `device` (about 0.3 s; allocates about 1.5 GiB for the
 * duration, synchronous; the device becomes current on the calling thread).
 * GCC_ERR_CUDA on a CUDA failure, GCC_ERR_DEVICE if a contended probe made
 * no progress or lost an update. */
gcc_status gcc_probe_memory(int device, gcc_memory_probe *out);

/* Message of the last failing call on this thread ("" if none). */
const char *gcc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GCC_GB300_H */
