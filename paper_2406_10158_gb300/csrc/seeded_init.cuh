// seeded_init.cuh -- seeded initial values of a key-value table's slots.
//
// Slot (key, field) of a table with n_fields fields takes output number
// key * n_fields + field + 1 of splitmix64 (Steele, Lea and Flood, 2014)
// seeded with `seed`.  A 16-byte slot holds a 10-byte value: that output in
// bytes 0-7, the low 16 bits of the same output number under the seed
// splitmix64(seed, 2) in bytes 8-9, and zeros in bytes 10-15.  The header is
// self-contained so that its host side also compiles as plain C++.
#pragma once

#include <cstdint>

#ifdef __CUDACC__
#define GCC_SEEDED_HD __host__ __device__
#else
#define GCC_SEEDED_HD
#endif

namespace gcc {
namespace seeded {

constexpr uint64_t GOLDEN = 0x9E3779B97F4A7C15ull;

// splitmix64's output function
GCC_SEEDED_HD inline uint64_t finalise(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// output number `counter` (1-based) of splitmix64 seeded with `seed`
GCC_SEEDED_HD inline uint64_t at(uint64_t seed, uint64_t counter) {
    return finalise(seed + GOLDEN * counter);
}

// bytes 0-7 of slot (key, field)
GCC_SEEDED_HD inline uint64_t slot_lo(uint64_t seed, uint64_t key, uint64_t field,
                                      uint64_t n_fields) {
    return at(seed, key * n_fields + field + 1);
}

// bytes 8-9 of a 16-byte slot, as the low 16 bits of a u64
GCC_SEEDED_HD inline uint64_t slot_hi(uint64_t seed, uint64_t key, uint64_t field,
                                      uint64_t n_fields) {
    return at(at(seed, 2), key * n_fields + field + 1) & 0xFFFFull;
}

}  // namespace seeded
}  // namespace gcc
