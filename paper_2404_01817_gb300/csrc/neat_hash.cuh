// Open-addressing hash tables in shared memory for key lookups inside one
// block: capacity a power of two at least twice the number of entries, so
// every probe sequence (linear probing) reaches a free slot.  Insertions use
// shared-memory atomics; lookups run after a barrier that follows the last
// insertion.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace neat {

constexpr unsigned long long kFree = ~0ull;

__device__ __forceinline__ uint32_t tslot(unsigned long long x, uint32_t mask)
{
    uint32_t h = (uint32_t)x * 0x9E3779B1u ^ (uint32_t)(x >> 32) * 0x85EBCA6Bu;
    h ^= h >> 15;
    return h & mask;
}

// Key -> lowest row holding it (entries key << 32 | row).  True when the key
// was already present: a duplicated key.
__device__ __forceinline__ bool key_insert(unsigned long long *tab, uint32_t mask, uint32_t key, uint32_t row)
{
    const unsigned long long v = ((unsigned long long)key << 32) | row;
    uint32_t s = tslot(key, mask);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long old = atomicCAS(tab + s, kFree, v);
        if (old == kFree) return false;
        if ((uint32_t)(old >> 32) == key) {
            atomicMin(tab + s, v);
            return true;
        }
        s = (s + 1u) & mask;
    }
    return false;
}

// Lowest row holding `key`, or -1 (after every insertion).
__device__ __forceinline__ int key_row(const unsigned long long *tab, uint32_t mask, uint32_t key)
{
    uint32_t s = tslot(key, mask);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long v = tab[s];
        if (v == kFree) return -1;
        if ((uint32_t)(v >> 32) == key) return (int)(uint32_t)v;
        s = (s + 1u) & mask;
    }
    return -1;
}

// Set of (in << 24 | out) pairs.  True when the pair was already present.
__device__ __forceinline__ bool pair_insert(unsigned long long *tab, uint32_t mask, unsigned long long pair)
{
    uint32_t s = tslot(pair, mask);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long old = atomicCAS(tab + s, kFree, pair);
        if (old == kFree) return false;
        if (old == pair) return true;
        s = (s + 1u) & mask;
    }
    return false;
}

// (in << 24 | out) pair -> lowest row holding it (entries pair << 13 | row,
// row < 8192).
__device__ __forceinline__ void pair_row_insert(unsigned long long *tab, uint32_t mask, unsigned long long pair,
                                                uint32_t row)
{
    const unsigned long long v = (pair << 13) | row;
    uint32_t s = tslot(pair, mask);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long old = atomicCAS(tab + s, kFree, v);
        if (old == kFree) return;
        if ((old >> 13) == pair) {
            atomicMin(tab + s, v);
            return;
        }
        s = (s + 1u) & mask;
    }
}

__device__ __forceinline__ int pair_row(const unsigned long long *tab, uint32_t mask, unsigned long long pair)
{
    uint32_t s = tslot(pair, mask);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long v = tab[s];
        if (v == kFree) return -1;
        if ((v >> 13) == pair) return (int)(v & 0x1fffu);
        s = (s + 1u) & mask;
    }
    return -1;
}

}  // namespace neat
