// oe_work.cuh -- the order-entry workload policy: the NewOrder and Payment
// procedures (Sec. IV-A names them as the TPC-C transactions studied; their
// arithmetic is this library's reading, documented in the C ABI header).
//
// Tables are int64 columns (table ids as in gcc_db_create).  Control words
// cover warehouse, district, customer and stock rows; the item table is never
// written, so item reads take no control word.  A committed NewOrder inserts
// its order, new-order flag and order lines at slots addressed by the order id
// it read from its district row; the district row's control word serialises
// order ids, so inserts never collide and need no control word either.
#pragma once

#include "exec_common.cuh"

namespace gcc {
namespace oe {

enum Col {
    W_YTD, W_TAX, D_YTD, D_TAX, D_NEXT_O_ID, C_BALANCE, C_YTD_PAYMENT, C_PAYMENT_CNT,
    C_DISCOUNT, I_PRICE, S_QUANTITY, S_YTD, S_ORDER_CNT, S_REMOTE_CNT, O_C_ID, O_OL_CNT,
    O_ALL_LOCAL, NO_FLAG, OL_I_ID, OL_SUPPLY_W_ID, OL_QUANTITY, OL_AMOUNT
};
constexpr uint32_t ITEMS = 100000, CUST = 3000, DIST = 10, LINES = 15;

struct OeWork {
    static constexpr int SCHEMA = GCC_SCHEMA_ORDER_ENTRY;

    static __device__ __forceinline__ uint64_t* col(const ExecArgs& a, int c) {
        return reinterpret_cast<uint64_t*>(a.cols[c]);
    }
    static __device__ __forceinline__ uint64_t get(const ExecArgs& a, int c, uint32_t row) {
        return ld_relaxed(col(a, c) + row);
    }
    static __device__ __forceinline__ void put(const ExecArgs& a, int c, uint64_t row, uint64_t v) {
        st_relaxed(col(a, c) + row, v);
    }
    static __device__ __forceinline__ bool valid_txn(const ExecArgs&, const gcc_txn& tx) {
        return tx.type == GCC_TXN_NEW_ORDER || tx.type == GCC_TXN_PAYMENT;
    }
    static __device__ __forceinline__ bool valid_op(const ExecArgs& a, uint64_t d) {
        if (op_kind(d) == GCC_OE_I_READ) return op_key(d) < ITEMS;
        return cc_record(d, SCHEMA, a.n_warehouses, NO_CC) != NO_CC;
    }
    // The fixed op layout of each procedure.
    static __device__ bool valid_shape(const ExecArgs&, const Stage& S, uint32_t n, uint32_t type) {
        if (type == GCC_TXN_PAYMENT)
            return n == 3 && op_kind(S.desc[0]) == GCC_OE_W_PAY &&
                   op_kind(S.desc[1]) == GCC_OE_D_PAY && op_kind(S.desc[2]) == GCC_OE_C_PAY;
        if (n < 5 || n > 3 + 2 * LINES || (n - 3) % 2) return false;
        if (op_kind(S.desc[0]) != GCC_OE_W_READ || op_kind(S.desc[1]) != GCC_OE_D_NEWORDER ||
            op_kind(S.desc[2]) != GCC_OE_C_READ)
            return false;
        for (uint32_t i = 3; i < n; ++i)
            if (op_kind(S.desc[i]) != ((i % 2) ? GCC_OE_I_READ : GCC_OE_S_NEWORDER)) return false;
        return true;
    }
    static __device__ __forceinline__ uint32_t rec(const ExecArgs& a, uint64_t d) {
        return cc_record(d, SCHEMA, a.n_warehouses, NO_CC);
    }
    static __device__ __forceinline__ bool writes(uint64_t d) { return kind_writes(op_kind(d)); }

    static __device__ ulonglong2 load(const ExecArgs& a, uint64_t d) {
        const uint32_t k = op_key(d);
        switch (op_kind(d)) {
            case GCC_OE_W_READ: return make_ulonglong2(get(a, W_TAX, k), 0ull);
            case GCC_OE_W_PAY: return make_ulonglong2(get(a, W_YTD, k), 0ull);
            case GCC_OE_D_NEWORDER: return make_ulonglong2(get(a, D_NEXT_O_ID, k), get(a, D_TAX, k));
            case GCC_OE_D_PAY: return make_ulonglong2(get(a, D_YTD, k), 0ull);
            case GCC_OE_C_READ: return make_ulonglong2(get(a, C_DISCOUNT, k), get(a, C_BALANCE, k));
            case GCC_OE_C_PAY: return make_ulonglong2(get(a, C_BALANCE, k), get(a, C_PAYMENT_CNT, k));
            case GCC_OE_I_READ: return make_ulonglong2(get(a, I_PRICE, k), 0ull);
            default: return make_ulonglong2(get(a, S_QUANTITY, k), get(a, S_ORDER_CNT, k));
        }
    }
    // New values of the columns `load` returned, for the writing kinds.
    static __device__ ulonglong2 compute(const ExecArgs&, uint64_t d, ulonglong2 old, ulonglong2 opd) {
        const int64_t h = (int64_t)opd.x;
        switch (op_kind(d)) {
            case GCC_OE_W_PAY:
            case GCC_OE_D_PAY: return make_ulonglong2((uint64_t)((int64_t)old.x + h), 0ull);
            case GCC_OE_D_NEWORDER: return make_ulonglong2(old.x + 1, old.y);
            case GCC_OE_C_PAY: return make_ulonglong2((uint64_t)((int64_t)old.x - h), old.y + 1);
            case GCC_OE_S_NEWORDER: {
                const int64_t q = (int64_t)old.x, qty = (int64_t)opd.x;
                const int64_t nq = q >= qty + 10 ? q - qty : q - qty + 91;
                return make_ulonglong2((uint64_t)nq, old.y + 1);
            }
            default: return old;
        }
    }
    // Install the new values; columns no op reads are updated relative to
    // their current value (the record is held exclusively here).
    static __device__ void store(const ExecArgs& a, uint64_t d, ulonglong2 v, uint64_t opidx) {
        const uint32_t k = op_key(d);
        switch (op_kind(d)) {
            case GCC_OE_W_PAY: put(a, W_YTD, k, v.x); break;
            case GCC_OE_D_PAY: put(a, D_YTD, k, v.x); break;
            case GCC_OE_D_NEWORDER: put(a, D_NEXT_O_ID, k, v.x); break;
            case GCC_OE_C_PAY: {
                const uint64_t h = a.operands[opidx].x;
                put(a, C_BALANCE, k, v.x);
                put(a, C_PAYMENT_CNT, k, v.y);
                put(a, C_YTD_PAYMENT, k, get(a, C_YTD_PAYMENT, k) + h);
                break;
            }
            case GCC_OE_S_NEWORDER: {
                const ulonglong2 o = a.operands[opidx];
                put(a, S_QUANTITY, k, v.x);
                put(a, S_ORDER_CNT, k, v.y);
                put(a, S_YTD, k, get(a, S_YTD, k) + o.x);
                put(a, S_REMOTE_CNT, k, get(a, S_REMOTE_CNT, k) + o.y);
                break;
            }
            default: break;
        }
    }
    // A committed NewOrder inserts its order, new-order flag and lines.
    static __device__ void commit_step(const ExecArgs& a, const Lane& L, const Stage& S, uint32_t,
                                       uint64_t first, uint32_t nops) {
        __syncwarp(L.gmask);
        insert_new_order(a, L.lig, L.G, L.gmask, first, nops,
                         [&](uint32_t j) { return S.desc[j]; },
                         [&](uint32_t j) { return S.oldv[j]; });
    }
    // The inserts of a committed NewOrder (nothing for a Payment), by the G
    // lanes of `gmask`: desc(j) and read(j) give op j's descriptor and the
    // value it read.  The order id is the district's next order id the
    // transaction read; an id outside the order slots sets the insert error.
    template <class Desc, class Read>
    static __device__ void insert_new_order(const ExecArgs& a, uint32_t lig, uint32_t G,
                                            unsigned gmask, uint64_t first, uint32_t nops,
                                            Desc desc, Read read) {
        if (op_kind(desc(0)) != GCC_OE_W_READ) return;             // Payment: nothing
        const int64_t o_id = (int64_t)read(1).x;
        const uint32_t dist = op_key(desc(1));
        if (o_id < 1 || (uint64_t)o_id > a.order_cap) {
            if (lig == 0) atomicOr(&a.st->error, GCC_DEVERR_INSERT);
            return;
        }
        const uint64_t slot = (uint64_t)dist * a.order_cap + (uint64_t)(o_id - 1);
        const uint32_t n_lines = (nops - 3) / 2;
        bool remote = false;
        for (uint32_t l = lig; l < n_lines; l += G) {
            const uint64_t s = desc(4 + 2 * l);
            const ulonglong2 opd = a.operands[first + 4 + 2 * l];
            const uint64_t ol = slot * LINES + l;
            put(a, OL_I_ID, ol, op_key(desc(3 + 2 * l)));
            put(a, OL_SUPPLY_W_ID, ol, op_key(s) / ITEMS);
            put(a, OL_QUANTITY, ol, opd.x);
            put(a, OL_AMOUNT, ol, (uint64_t)((int64_t)opd.x * (int64_t)read(3 + 2 * l).x));
            if (opd.y) remote = true;
        }
        remote = __any_sync(gmask, remote);
        if (lig == 0) {
            put(a, O_C_ID, slot, op_key(desc(2)) % CUST);
            put(a, O_OL_CNT, slot, n_lines);
            put(a, O_ALL_LOCAL, slot, remote ? 0ull : 1ull);
            put(a, NO_FLAG, slot, 1ull);
        }
    }
};

}  // namespace oe
}  // namespace gcc
