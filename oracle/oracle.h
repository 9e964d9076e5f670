/*
 * oracle.h -- plain, single-threaded CPU oracle for batched OLTP execution.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this code; only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code with the CUDA engine.
 *
 * What it computes.  Every scheme the engine implements promises serializable
 * executions (Sec. III-E: all schemes ensure the serializable isolation level;
 * the isolation property is stated in Sec. II).  The engine reports, for each
 * transaction, whether it committed and its position in a commit order.  The
 * oracle starts from the same initial database, applies the committed
 * transactions one at a time in that reported order, records every value read,
 * and compares read values and final database with the engine's, word by word.
 * It also runs batches serially in any order given (transaction-id order is the
 * deterministic scheme's order, Sec. II-C), and, for batches of at most 8
 * transactions, enumerates all serial orders (brute force).
 *
 * Operation semantics (the paper leaves them open; these are the readings this
 * library fixes):
 *   key-value tables are field-major; a slot is 8 bytes (u64) or 16 bytes
 *   (u64 lo = bytes 0-7, u64 hi = bytes 8-15, payload in bytes 0-9);
 *   READ returns the slot; ADD returns the old slot and then adds the operand:
 *   8-byte slots wrap modulo 2^64; 16-byte slots add lo modulo 2^64 and bytes
 *   8-9 as a u16 modulo 2^16, bytes 10-15 unchanged.
 *   Order-entry procedures are described beside their functions below.
 *
 * Parity pins (see tests/test_oracle.py): closed forms (a single hot key's
 * reads are prefix sums of the deltas in commit order), read-only batches,
 * order independence of disjoint batches, conservation of the table sum,
 * hand-computed golden fixtures and brute force over all serial orders.
 */
#ifndef GCC_ORACLE_H
#define GCC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_BAD_KEY = 1, ORC_BAD_FIELD = 2, ORC_BAD_KIND = 3,
       ORC_BAD_ORDER = 4, ORC_TOO_MANY = 5, ORC_NOMEM = 6, ORC_BAD_TYPE = 7,
       ORC_NOT_COMMITTED = 8, ORC_BAD_INSERT = 9 };

/* op kinds */
enum { ORC_READ = 0, ORC_ADD = 1,
       /* order-entry op kinds */
       ORC_OE_W_READ = 16, ORC_OE_W_PAY = 17, ORC_OE_D_NEWORDER = 18,
       ORC_OE_D_PAY = 19, ORC_OE_C_READ = 20, ORC_OE_C_PAY = 21,
       ORC_OE_I_READ = 22, ORC_OE_S_NEWORDER = 23, ORC_OE_C_PAY_BY_NAME = 24 };

/* transaction types */
enum { ORC_TXN_KV = 0, ORC_TXN_NEW_ORDER = 1, ORC_TXN_PAYMENT = 2 };

/* per-transaction status values reported by the engine */
enum { ORC_ST_PENDING = 0, ORC_ST_COMMITTED = 1, ORC_ST_TIMEOUT = 2, ORC_ST_INVALID = 3 };

typedef struct { uint32_t first_op; uint16_t n_ops; uint16_t type; } orc_txn;
typedef struct { uint32_t key; uint8_t field; uint8_t kind; uint16_t aux; } orc_op;
typedef struct { uint32_t status; uint32_t attempts; uint64_t commit_order; } orc_result;

/* A key-value table: field-major, nfields x nrec slots of field_bytes (8|16). */
typedef struct {
    uint64_t *table;
    uint64_t nrec;
    uint32_t nfields;
    uint32_t field_bytes;
} orc_kv;

typedef struct {
    int32_t err;                 /* ORC_* code of the first structural error */
    uint32_t n_committed;
    uint64_t n_read_mismatch;    /* read values that differ */
    uint64_t first_bad_op;       /* op index of the first differing read (or ~0) */
    uint64_t n_table_mismatch;   /* 64-bit words of the final database that differ */
    uint64_t first_bad_word;     /* index of the first differing word (or ~0) */
} orc_report;

/* Execute transaction t serially on db.  reads (2 u64 per op, indexed by the
 * global op index) receives the value each op read; may be NULL. */
int orc_kv_run_txn(orc_kv *db, const orc_txn *t, const orc_op *ops,
                   const uint64_t *operands, uint64_t *reads);

/* Execute txns[order[0]], txns[order[1]], ... serially; order == NULL means
 * transaction-id order over all n_txns. */
int orc_kv_serial(orc_kv *db, const orc_txn *txns, uint32_t n_txns,
                  const orc_op *ops, const uint64_t *operands,
                  const uint32_t *order, uint32_t n_order, uint64_t *reads);

/* From per-transaction results, the sequence of committed transaction ids in
 * commit order.  Fails with ORC_BAD_ORDER unless the committed transactions'
 * commit_order values are exactly a permutation of 0..n_committed-1. */
int orc_commit_sequence(const orc_result *res, uint32_t n_txns,
                        uint32_t *order, uint32_t *n_committed);

/* Replay the committed transactions in their reported commit order on `work`
 * (which must hold the initial database and is modified), then compare reads
 * of committed transactions with gpu_reads and the final table with gpu_table.
 * With require_all != 0, a transaction that did not commit is an error. */
int orc_kv_replay_check(orc_kv *work, const uint64_t *gpu_table,
                        const orc_txn *txns, uint32_t n_txns,
                        const orc_op *ops, const uint64_t *operands,
                        const orc_result *res, const uint64_t *gpu_reads,
                        int require_all, orc_report *rep);

/* Brute force over all n_txns! serial orders (n_txns <= 8): the number of
 * orders whose reads and final table equal obs_reads / obs_table.  The first
 * matching order is written to first_match (may be NULL).  Negative = error. */
int64_t orc_kv_brute_force(const orc_kv *init, const orc_txn *txns, uint32_t n_txns,
                           const orc_op *ops, const uint64_t *operands,
                           const uint64_t *obs_reads, const uint64_t *obs_table,
                           uint32_t *first_match);

/* Sum of all slots: per 64-bit lane for 16-byte slots (lane 1 summed as the
 * u16 in bytes 8-9 modulo 2^16); out[0] = lane 0, out[1] = lane 1. */
void orc_kv_sum(const orc_kv *db, uint64_t out[2]);

/* ---------------------------------------------------------------------------
 * Order-entry schema (TPC-C-like NewOrder and Payment, Sec. IV-A; the paper
 * names the transactions only).  Columns are int64 arrays; see oracle.c.
 * ------------------------------------------------------------------------- */
typedef struct {
    uint32_t W;                    /* warehouses */
    uint32_t order_cap;            /* order slots per district */
    /* warehouse [W] */
    int64_t *w_ytd, *w_tax;
    /* district [10W] */
    int64_t *d_ytd, *d_tax, *d_next_o_id;
    /* customer [30000W] */
    int64_t *c_balance, *c_ytd_payment, *c_payment_cnt, *c_discount;
    /* item [100000] */
    int64_t *i_price;
    /* stock [100000W] */
    int64_t *s_quantity, *s_ytd, *s_order_cnt, *s_remote_cnt;
    /* order [10W * order_cap] */
    int64_t *o_c_id, *o_ol_cnt, *o_all_local;
    /* new-order flag [10W * order_cap] */
    int64_t *no_flag;
    /* order-line [10W * order_cap * 15] */
    int64_t *ol_i_id, *ol_supply_w_id, *ol_quantity, *ol_amount;
    /* customer names [30000W], never written: last-name id, first-name key */
    int64_t *c_last, *c_first;
} orc_oe;

int orc_oe_run_txn(orc_oe *db, const orc_txn *t, const orc_op *ops,
                   const uint64_t *operands, uint64_t *reads);
int orc_oe_serial(orc_oe *db, const orc_txn *txns, uint32_t n_txns,
                  const orc_op *ops, const uint64_t *operands,
                  const uint32_t *order, uint32_t n_order, uint64_t *reads);
/* Consistency conditions of the order-entry state (0 = all hold):
 * bit 0: for every district, d_next_o_id - 1 equals the largest order id
 *        present and the largest new-order id present;
 * bit 1: for every warehouse, w_ytd equals the sum of its districts' d_ytd;
 * bit 2: every present order has exactly o_ol_cnt order lines present. */
int orc_oe_check_consistency(const orc_oe *db);

#ifdef __cplusplus
}
#endif
#endif
