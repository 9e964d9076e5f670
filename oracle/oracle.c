/*
 * oracle.c -- plain serial executor, replay checker and brute force.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Deliberately simple: one
 * transaction at a time, one op at a time, no blocking, no reordering.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* key-value tables                                                          */
/* ------------------------------------------------------------------------ */

/* Address of the slot (key, field) in a field-major table. */
static uint64_t *kv_slot(orc_kv *db, uint32_t key, uint32_t field)
{
    uint64_t words = db->field_bytes / 8;
    return db->table + ((uint64_t)field * db->nrec + key) * words;
}

/* Apply one op; out[0..1] receives the value read (the slot before the op). */
static int kv_apply_op(orc_kv *db, const orc_op *op, const uint64_t *operand,
                       uint64_t out[2])
{
    if (op->key >= db->nrec) return ORC_BAD_KEY;
    if (op->field >= db->nfields) return ORC_BAD_FIELD;
    uint64_t *s = kv_slot(db, op->key, op->field);
    uint64_t old_lo = s[0];
    uint64_t old_hi = (db->field_bytes == 16) ? s[1] : 0;
    if (op->kind == ORC_READ) {
        /* a read leaves the record unchanged */
    } else if (op->kind == ORC_ADD) {
        s[0] = old_lo + operand[0];                        /* mod 2^64 */
        if (db->field_bytes == 16) {
            uint64_t b89 = (old_hi + operand[1]) & 0xFFFFull;
            s[1] = (old_hi & ~0xFFFFull) | b89;            /* bytes 10-15 kept */
        }
    } else {
        return ORC_BAD_KIND;
    }
    out[0] = old_lo;
    out[1] = old_hi;
    return ORC_OK;
}

int orc_kv_run_txn(orc_kv *db, const orc_txn *t, const orc_op *ops,
                   const uint64_t *operands, uint64_t *reads)
{
    if (t->type != ORC_TXN_KV)
        return ORC_BAD_TYPE;
    for (uint32_t i = 0; i < t->n_ops; i++) {
        uint64_t g = (uint64_t)t->first_op + i;     /* global op index */
        uint64_t got[2];
        int e = kv_apply_op(db, &ops[g], &operands[2 * g], got);
        if (e) return e;
        if (reads) {
            reads[2 * g] = got[0];
            reads[2 * g + 1] = got[1];
        }
    }
    return ORC_OK;
}

int orc_kv_serial(orc_kv *db, const orc_txn *txns, uint32_t n_txns,
                  const orc_op *ops, const uint64_t *operands,
                  const uint32_t *order, uint32_t n_order, uint64_t *reads)
{
    uint32_t n = order ? n_order : n_txns;
    for (uint32_t k = 0; k < n; k++) {
        uint32_t tid = order ? order[k] : k;
        if (tid >= n_txns) return ORC_BAD_ORDER;
        int e = orc_kv_run_txn(db, &txns[tid], ops, operands, reads);
        if (e) return e;
    }
    return ORC_OK;
}

int orc_commit_sequence(const orc_result *res, uint32_t n_txns,
                        uint32_t *order, uint32_t *n_committed)
{
    uint32_t nc = 0;
    for (uint32_t t = 0; t < n_txns; t++)
        if (res[t].status == ORC_ST_COMMITTED) nc++;
    for (uint32_t k = 0; k < nc; k++) order[k] = UINT32_MAX;
    for (uint32_t t = 0; t < n_txns; t++) {
        if (res[t].status != ORC_ST_COMMITTED) continue;
        uint64_t pos = res[t].commit_order;
        if (pos >= nc || order[pos] != UINT32_MAX) {
            *n_committed = nc;
            return ORC_BAD_ORDER;                 /* not a permutation */
        }
        order[pos] = t;
    }
    *n_committed = nc;
    return ORC_OK;
}

static uint64_t kv_words(const orc_kv *db)
{
    return db->nrec * db->nfields * (db->field_bytes / 8);
}

static void note_read(orc_report *rep, uint64_t g, const uint64_t mine[2],
                      const uint64_t *gpu_reads)
{
    if (mine[0] != gpu_reads[2 * g] || mine[1] != gpu_reads[2 * g + 1]) {
        if (rep->n_read_mismatch == 0) rep->first_bad_op = g;
        rep->n_read_mismatch++;
    }
}

static void compare_words(orc_report *rep, const uint64_t *a, const uint64_t *b,
                          uint64_t n, uint64_t offset)
{
    for (uint64_t i = 0; i < n; i++) {
        if (a[i] != b[i]) {
            if (rep->n_table_mismatch == 0) rep->first_bad_word = offset + i;
            rep->n_table_mismatch++;
        }
    }
}

int orc_kv_replay_check(orc_kv *work, const uint64_t *gpu_table,
                        const orc_txn *txns, uint32_t n_txns,
                        const orc_op *ops, const uint64_t *operands,
                        const orc_result *res, const uint64_t *gpu_reads,
                        int require_all, orc_report *rep)
{
    memset(rep, 0, sizeof *rep);
    rep->first_bad_op = ~0ull;
    rep->first_bad_word = ~0ull;
    uint32_t *order = malloc(sizeof(uint32_t) * (n_txns ? n_txns : 1));
    if (!order) return rep->err = ORC_NOMEM;
    uint32_t nc = 0;
    int e = orc_commit_sequence(res, n_txns, order, &nc);
    rep->n_committed = nc;
    if (!e && require_all && nc != n_txns) e = ORC_NOT_COMMITTED;

    /* replay the committed transactions in commit order */
    for (uint32_t k = 0; !e && k < nc; k++) {
        const orc_txn *t = &txns[order[k]];
        if (t->type != ORC_TXN_KV) { e = ORC_BAD_TYPE; break; }
        for (uint32_t i = 0; i < t->n_ops; i++) {
            uint64_t g = (uint64_t)t->first_op + i;
            uint64_t mine[2];
            e = kv_apply_op(work, &ops[g], &operands[2 * g], mine);
            if (e) break;
            note_read(rep, g, mine, gpu_reads);
        }
    }
    free(order);
    if (e) return rep->err = e;
    compare_words(rep, work->table, gpu_table, kv_words(work), 0);
    return rep->err = ORC_OK;
}

/* Next permutation in lexicographic order; 0 when `p` was the last one. */
static int next_permutation(uint32_t *p, uint32_t n)
{
    if (n < 2) return 0;
    int i = (int)n - 2;
    while (i >= 0 && p[i] >= p[i + 1]) i--;
    if (i < 0) return 0;
    int j = (int)n - 1;
    while (p[j] <= p[i]) j--;
    uint32_t tmp = p[i]; p[i] = p[j]; p[j] = tmp;
    for (int a = i + 1, b = (int)n - 1; a < b; a++, b--) {
        tmp = p[a]; p[a] = p[b]; p[b] = tmp;
    }
    return 1;
}

int64_t orc_kv_brute_force(const orc_kv *init, const orc_txn *txns, uint32_t n_txns,
                           const orc_op *ops, const uint64_t *operands,
                           const uint64_t *obs_reads, const uint64_t *obs_table,
                           uint32_t *first_match)
{
    if (n_txns > 8) return -ORC_TOO_MANY;
    uint64_t words = kv_words(init);
    uint64_t n_ops = 0;
    for (uint32_t t = 0; t < n_txns; t++) {
        uint64_t end = (uint64_t)txns[t].first_op + txns[t].n_ops;
        if (end > n_ops) n_ops = end;
    }
    uint64_t *table = malloc(sizeof(uint64_t) * (words ? words : 1));
    uint64_t *reads = calloc(2 * (n_ops ? n_ops : 1), sizeof(uint64_t));
    if (!table || !reads) { free(table); free(reads); return -ORC_NOMEM; }
    uint32_t perm[8];
    for (uint32_t k = 0; k < n_txns; k++) perm[k] = k;
    int64_t matches = 0;
    do {
        memcpy(table, init->table, sizeof(uint64_t) * words);
        orc_kv db = *init;
        db.table = table;
        int e = orc_kv_serial(&db, txns, n_txns, ops, operands, perm, n_txns, reads);
        if (e) { matches = -e; break; }
        int same = memcmp(table, obs_table, sizeof(uint64_t) * words) == 0;
        for (uint32_t t = 0; same && t < n_txns; t++)
            for (uint32_t i = 0; same && i < txns[t].n_ops; i++) {
                uint64_t g = (uint64_t)txns[t].first_op + i;
                same = reads[2 * g] == obs_reads[2 * g] &&
                       reads[2 * g + 1] == obs_reads[2 * g + 1];
            }
        if (same) {
            if (matches == 0 && first_match)
                memcpy(first_match, perm, sizeof(uint32_t) * n_txns);
            matches++;
        }
    } while (next_permutation(perm, n_txns));
    free(table);
    free(reads);
    return matches;
}

void orc_kv_sum(const orc_kv *db, uint64_t out[2])
{
    uint64_t s0 = 0, s1 = 0;
    uint64_t slots = db->nrec * db->nfields;
    if (db->field_bytes == 16) {
        for (uint64_t i = 0; i < slots; i++) {
            s0 += db->table[2 * i];
            s1 = (s1 + (db->table[2 * i + 1] & 0xFFFFull)) & 0xFFFFull;
        }
    } else {
        for (uint64_t i = 0; i < slots; i++) s0 += db->table[i];
    }
    out[0] = s0;
    out[1] = s1;
}

/* ------------------------------------------------------------------------ */
/* order-entry schema                                                        */
/*                                                                           */
/* Rows: warehouse w in [0,W); district w*10+d; customer (w*10+d)*3000+c;    */
/* item i in [0,100000); stock w*100000+i; order slot                        */
/* (w*10+d)*order_cap + (o_id-1); order line (order slot)*15 + line.         */
/*                                                                           */
/* NewOrder ops, in procedure order:                                         */
/*   0 W_READ     key w           reads (w_tax, 0)                           */
/*   1 D_NEWORDER key district    reads (d_next_o_id, d_tax); next_o_id += 1 */
/*   2 C_READ     key customer    reads (c_discount, c_balance)              */
/*   then per order line l = 0..ol_cnt-1:                                    */
/*   3+2l I_READ     key item         reads (i_price, 0)                     */
/*   4+2l S_NEWORDER key stock row    operand (qty, remote)                  */
/*        reads (s_quantity, s_order_cnt); s_quantity -= qty, plus 91 when   */
/*        the old quantity was below qty + 10; s_ytd += qty;                 */
/*        s_order_cnt += 1; s_remote_cnt += remote                           */
/*   at commit: order o_id = d_next_o_id read by op 1 is inserted with       */
/*   o_c_id, o_ol_cnt, o_all_local, a new-order flag and its order lines     */
/*   (item, supply warehouse, quantity, amount = quantity * i_price).        */
/* Payment ops:                                                              */
/*   0 W_PAY  key w        operand h   reads (w_ytd, 0);  w_ytd += h         */
/*   1 D_PAY  key district operand h   reads (d_ytd, 0);  d_ytd += h         */
/*   2 C_PAY  key customer operand h   reads (c_balance, c_payment_cnt);     */
/*        c_balance -= h; c_ytd_payment += h; c_payment_cnt += 1             */
/*     or C_PAY_BY_NAME key district, aux last-name id, operand h: the       */
/*        customer of that district chosen by name (oe_customer_by_name),    */
/*        then as C_PAY                                                      */
/* ------------------------------------------------------------------------ */
enum { OE_ITEMS = 100000, OE_CUST = 3000, OE_DIST = 10, OE_LINES = 15 };

/* Payment by last name: among the district's customers whose last name is
 * `name`, ordered by first name and then by customer index, the one at
 * position ceil(n/2) (1-based).  Returns the customer's row, or -1 when
 * nobody in the district has the name.  (The paper names the payment
 * transaction only, Sec. IV-A; this selection rule is the library's reading.) */
static int64_t oe_customer_by_name(const orc_oe *db, uint64_t district, int64_t name)
{
    uint64_t base = district * OE_CUST;
    int64_t n = 0;
    for (uint64_t c = 0; c < OE_CUST; c++)
        if (db->c_last[base + c] == name) n++;
    if (n == 0) return -1;
    int64_t want = (n + 1) / 2 - 1;          /* 0-based position of ceil(n/2) */
    for (uint64_t c = 0; c < OE_CUST; c++) {
        if (db->c_last[base + c] != name) continue;
        int64_t before = 0;                  /* named customers ordered before c */
        for (uint64_t o = 0; o < OE_CUST; o++) {
            if (db->c_last[base + o] != name) continue;
            if (db->c_first[base + o] < db->c_first[base + c] ||
                (db->c_first[base + o] == db->c_first[base + c] && o < c))
                before++;
        }
        if (before == want) return (int64_t)(base + c);
    }
    return -1;
}

static int oe_apply_op(orc_oe *db, const orc_op *op, const uint64_t *operand,
                       uint64_t out[2])
{
    uint64_t W = db->W;
    uint32_t k = op->key;
    out[0] = out[1] = 0;
    switch (op->kind) {
    case ORC_OE_W_READ:
        if (k >= W) return ORC_BAD_KEY;
        out[0] = (uint64_t)db->w_tax[k];
        return ORC_OK;
    case ORC_OE_W_PAY:
        if (k >= W) return ORC_BAD_KEY;
        out[0] = (uint64_t)db->w_ytd[k];
        db->w_ytd[k] += (int64_t)operand[0];
        return ORC_OK;
    case ORC_OE_D_NEWORDER:
        if (k >= W * OE_DIST) return ORC_BAD_KEY;
        out[0] = (uint64_t)db->d_next_o_id[k];
        out[1] = (uint64_t)db->d_tax[k];
        db->d_next_o_id[k] += 1;
        return ORC_OK;
    case ORC_OE_D_PAY:
        if (k >= W * OE_DIST) return ORC_BAD_KEY;
        out[0] = (uint64_t)db->d_ytd[k];
        db->d_ytd[k] += (int64_t)operand[0];
        return ORC_OK;
    case ORC_OE_C_READ:
        if (k >= W * OE_DIST * OE_CUST) return ORC_BAD_KEY;
        out[0] = (uint64_t)db->c_discount[k];
        out[1] = (uint64_t)db->c_balance[k];
        return ORC_OK;
    case ORC_OE_C_PAY_BY_NAME:
    case ORC_OE_C_PAY: {
        if (op->kind == ORC_OE_C_PAY_BY_NAME) {
            if (k >= W * OE_DIST) return ORC_BAD_KEY;
            int64_t row = oe_customer_by_name(db, k, (int64_t)op->aux);
            if (row < 0) return ORC_BAD_KEY;
            k = (uint32_t)row;
        }
        if (k >= W * OE_DIST * OE_CUST) return ORC_BAD_KEY;
        int64_t h = (int64_t)operand[0];
        out[0] = (uint64_t)db->c_balance[k];
        out[1] = (uint64_t)db->c_payment_cnt[k];
        db->c_balance[k] -= h;
        db->c_ytd_payment[k] += h;
        db->c_payment_cnt[k] += 1;
        return ORC_OK;
    }
    case ORC_OE_I_READ:
        if (k >= OE_ITEMS) return ORC_BAD_KEY;
        out[0] = (uint64_t)db->i_price[k];
        return ORC_OK;
    case ORC_OE_S_NEWORDER: {
        if (k >= W * OE_ITEMS) return ORC_BAD_KEY;
        int64_t qty = (int64_t)operand[0];
        int64_t remote = (int64_t)operand[1];
        int64_t q = db->s_quantity[k];
        out[0] = (uint64_t)q;
        out[1] = (uint64_t)db->s_order_cnt[k];
        if (q >= qty + 10)
            db->s_quantity[k] = q - qty;
        else
            db->s_quantity[k] = q - qty + 91;
        db->s_ytd[k] += qty;
        db->s_order_cnt[k] += 1;
        db->s_remote_cnt[k] += remote;
        return ORC_OK;
    }
    default:
        return ORC_BAD_KIND;
    }
}

/* The rows a committed NewOrder inserts (order, new-order flag, lines). */
static int oe_insert_order(orc_oe *db, const orc_txn *t, const orc_op *ops,
                           const uint64_t *operands, const uint64_t *reads)
{
    uint64_t f = t->first_op;
    uint32_t n_lines = (uint32_t)(t->n_ops - 3) / 2;
    uint32_t dist = ops[f + 1].key;
    int64_t o_id = (int64_t)reads[2 * 1];
    if (o_id < 1 || (uint64_t)o_id > db->order_cap) return ORC_BAD_INSERT;
    uint64_t slot = (uint64_t)dist * db->order_cap + (uint64_t)(o_id - 1);
    uint32_t cust = ops[f + 2].key;
    int64_t all_local = 1;
    for (uint32_t l = 0; l < n_lines; l++) {
        uint64_t s = f + 4 + 2 * l;
        uint64_t ol = slot * OE_LINES + l;
        uint32_t item = ops[f + 3 + 2 * l].key;
        int64_t qty = (int64_t)operands[2 * s];
        int64_t price = (int64_t)reads[2 * (3 + 2 * l)];
        if (operands[2 * s + 1]) all_local = 0;
        db->ol_i_id[ol] = item;
        db->ol_supply_w_id[ol] = ops[s].key / OE_ITEMS;
        db->ol_quantity[ol] = qty;
        db->ol_amount[ol] = qty * price;
    }
    db->o_c_id[slot] = cust % OE_CUST;
    db->o_ol_cnt[slot] = n_lines;
    db->o_all_local[slot] = all_local;
    db->no_flag[slot] = 1;
    return ORC_OK;
}

/* Run one order-entry transaction; reads (2 u64 per op) are indexed by the
 * global op index and may be NULL. */
int orc_oe_run_txn(orc_oe *db, const orc_txn *t, const orc_op *ops,
                   const uint64_t *operands, uint64_t *reads)
{
    uint64_t local[2 * (3 + 2 * OE_LINES)];
    uint64_t f = t->first_op;
    if (t->type == ORC_TXN_NEW_ORDER) {
        if (t->n_ops < 5 || t->n_ops > 3 + 2 * OE_LINES || (t->n_ops - 3) % 2)
            return ORC_BAD_TYPE;
        static const uint8_t head[3] = { ORC_OE_W_READ, ORC_OE_D_NEWORDER, ORC_OE_C_READ };
        for (uint32_t i = 0; i < 3; i++)
            if (ops[f + i].kind != head[i]) return ORC_BAD_KIND;
        for (uint32_t i = 3; i < t->n_ops; i++)
            if (ops[f + i].kind != ((i % 2) ? ORC_OE_I_READ : ORC_OE_S_NEWORDER))
                return ORC_BAD_KIND;
    } else if (t->type == ORC_TXN_PAYMENT) {
        if (t->n_ops != 3 || ops[f].kind != ORC_OE_W_PAY ||
            ops[f + 1].kind != ORC_OE_D_PAY ||
            (ops[f + 2].kind != ORC_OE_C_PAY && ops[f + 2].kind != ORC_OE_C_PAY_BY_NAME))
            return ORC_BAD_KIND;
    } else {
        return ORC_BAD_TYPE;
    }
    for (uint32_t i = 0; i < t->n_ops; i++) {
        int e = oe_apply_op(db, &ops[f + i], &operands[2 * (f + i)], &local[2 * i]);
        if (e) return e;
    }
    if (t->type == ORC_TXN_NEW_ORDER) {
        int e = oe_insert_order(db, t, ops, operands, local);
        if (e) return e;
    }
    if (reads)
        memcpy(&reads[2 * f], local, sizeof(uint64_t) * 2 * t->n_ops);
    return ORC_OK;
}

int orc_oe_serial(orc_oe *db, const orc_txn *txns, uint32_t n_txns,
                  const orc_op *ops, const uint64_t *operands,
                  const uint32_t *order, uint32_t n_order, uint64_t *reads)
{
    uint32_t n = order ? n_order : n_txns;
    for (uint32_t k = 0; k < n; k++) {
        uint32_t tid = order ? order[k] : k;
        if (tid >= n_txns) return ORC_BAD_ORDER;
        int e = orc_oe_run_txn(db, &txns[tid], ops, operands, reads);
        if (e) return e;
    }
    return ORC_OK;
}

int orc_oe_check_consistency(const orc_oe *db)
{
    int bad = 0;
    uint64_t nd = (uint64_t)db->W * OE_DIST;
    for (uint64_t d = 0; d < nd; d++) {
        int64_t max_o = 0, max_no = 0;
        for (uint64_t o = 0; o < db->order_cap; o++) {
            uint64_t slot = d * db->order_cap + o;
            if (db->o_ol_cnt[slot] > 0) max_o = (int64_t)o + 1;
            if (db->no_flag[slot]) max_no = (int64_t)o + 1;
            int64_t cnt = db->o_ol_cnt[slot];
            for (int64_t l = 0; l < OE_LINES; l++) {
                int present = db->ol_quantity[slot * OE_LINES + l] > 0;
                if (present != (l < cnt)) bad |= 4;
            }
        }
        if (max_o != db->d_next_o_id[d] - 1 || max_no != db->d_next_o_id[d] - 1)
            bad |= 1;
    }
    for (uint64_t w = 0; w < db->W; w++) {
        int64_t s = 0;
        for (uint64_t d = 0; d < OE_DIST; d++) s += db->d_ytd[w * OE_DIST + d];
        if (s != db->w_ytd[w]) bad |= 2;
    }
    return bad;
}
