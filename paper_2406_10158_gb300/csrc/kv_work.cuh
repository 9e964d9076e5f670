// kv_work.cuh -- the key-value workload policy of the execute kernels.
//
// One table of n_records x n_fields slots, field-major ("columnar"): slot
// (key, field) at byte (field * n_records + key) * FB, FB = 8 or 16.  One
// control word per record (conflicts at record granularity).  READ returns the
// slot; ADD returns the old slot and adds the operand -- 8-byte slots modulo
// 2^64; 16-byte slots lane 0 modulo 2^64 and bytes 8-9 as a u16 modulo 2^16,
// bytes 10-15 kept.  16-byte slots move as one vector load / store.
#pragma once

#include "exec_common.cuh"

namespace gcc {

template <int FB> struct Slot;

template <> struct Slot<8> {
    static __device__ __forceinline__ ulonglong2 load(const uint8_t* p) {
        return make_ulonglong2(ld_relaxed(reinterpret_cast<const uint64_t*>(p)), 0ull);
    }
    static __device__ __forceinline__ void store(uint8_t* p, ulonglong2 v) {
        st_relaxed(reinterpret_cast<uint64_t*>(p), v.x);
    }
    static __device__ __forceinline__ ulonglong2 add(ulonglong2 v, ulonglong2 d) {
        return make_ulonglong2(v.x + d.x, 0ull);
    }
};

template <> struct Slot<16> {
    static __device__ __forceinline__ ulonglong2 load(const uint8_t* p) { return ld_slot16(p); }
    static __device__ __forceinline__ void store(uint8_t* p, ulonglong2 v) { st_slot16(p, v); }
    static __device__ __forceinline__ ulonglong2 add(ulonglong2 v, ulonglong2 d) {
        return make_ulonglong2(v.x + d.x, (v.y & ~0xFFFFull) | ((v.y + d.y) & 0xFFFFull));
    }
};

template <int FB>
struct KvWork {
    static constexpr int SCHEMA = GCC_SCHEMA_KV;

    static __device__ __forceinline__ uint8_t* ptr(const ExecArgs& a, uint64_t d) {
        return a.table + ((uint64_t)op_field(d) * a.n_records + op_key(d)) * FB;
    }
    static __device__ __forceinline__ bool valid_txn(const ExecArgs&, const gcc_txn& tx) {
        return tx.type == GCC_TXN_KV;
    }
    static __device__ __forceinline__ bool valid_op(const ExecArgs& a, uint64_t d) {
        return op_key(d) < a.n_records && op_field(d) < a.n_fields &&
               (op_kind(d) == GCC_OP_READ || op_kind(d) == GCC_OP_ADD);
    }
    static __device__ __forceinline__ bool valid_shape(const ExecArgs&, const Stage&, uint32_t,
                                                       uint32_t) {
        return true;
    }
    static __device__ __forceinline__ uint32_t rec(const ExecArgs&, uint64_t d) { return op_key(d); }
    static __device__ __forceinline__ bool writes(uint64_t d) { return op_kind(d) == GCC_OP_ADD; }
    static __device__ __forceinline__ ulonglong2 load(const ExecArgs& a, uint64_t d) {
        return Slot<FB>::load(ptr(a, d));
    }
    static __device__ __forceinline__ ulonglong2 compute(const ExecArgs&, uint64_t, ulonglong2 old,
                                                         ulonglong2 operand) {
        return Slot<FB>::add(old, operand);
    }
    static __device__ __forceinline__ void store(const ExecArgs& a, uint64_t d, ulonglong2 v,
                                                 uint64_t) {
        Slot<FB>::store(ptr(a, d), v);
    }
    static __device__ __forceinline__ void commit_step(const ExecArgs&, const Lane&, const Stage&,
                                                       uint32_t, uint64_t, uint32_t) {}
};

}  // namespace gcc
