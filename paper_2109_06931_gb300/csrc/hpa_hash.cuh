// Open-addressing hash tables of 64-bit keys with a 32-bit value per slot,
// for grouping equal keys on the device: insertion claims a slot with a
// compare-and-swap on the key and keeps the minimum of the inserted values
// (the representative: the first index, in input order, with that key); a
// second pass reads the representative from the slot the insertion returned.
// Linear probing; tables hold a power of two of slots, at least twice the
// keys inserted, keys initialised to all ones (which no key may equal) and
// values to all ones.
#pragma once

#include <cstdint>

namespace hpa {

constexpr unsigned long long UEMPTY = ~0ull;

// slot of a key: the 64-bit finalizer of MurmurHash3 (Appleby), masked
__device__ __forceinline__ uint32_t uhash(unsigned long long k, uint32_t mask) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return (uint32_t)k & mask;
}

// Returns the key's slot, or 0xFFFFFFFF when the table is full; once every
// insertion has finished, vals[slot] is the key's representative.
__device__ __forceinline__ uint32_t ut_insert(unsigned long long* keys, uint32_t* vals, uint32_t mask,
                                              unsigned long long key, uint32_t idx) {
    uint32_t h = uhash(key, mask);
    volatile unsigned long long* vk = keys;
    for (uint32_t t = 0; t <= mask; ++t) {
        unsigned long long cur = vk[h];
        if (cur == UEMPTY) {
            cur = atomicCAS(&keys[h], UEMPTY, key);
            if (cur == UEMPTY) cur = key;
        }
        if (cur == key) { atomicMin(&vals[h], idx); return h; }
        h = (h + 1) & mask;
    }
    return 0xFFFFFFFFu;
}

}  // namespace hpa
