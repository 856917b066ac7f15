// bounds.cuh -- range checks of the kernels' global-memory indices in the
// debug build (compiled with -DSPINSIM_BOUNDS; see build.build_bounds).
//
// SPINSIM_INB(cond, bit) is true when cond holds.  In the debug build a
// failed check sets bit `bit` of the translation unit's device error word and
// yields false, and the caller skips the access (it never traps, asserts or
// returns early, so warp- and block-wide synchronisation is unaffected); the
// host reads and clears the words with spinsim_debug_bounds.  In the normal
// build the check is the constant true and compiles away.
#pragma once
#include <cstdint>

#ifdef SPINSIM_BOUNDS
static __device__ unsigned long long g_spinsim_bounds_word;
__device__ __forceinline__ bool spinsim_bounds_fail(int bit)
{
    atomicOr(&g_spinsim_bounds_word, 1ULL << bit);
    return false;
}
#define SPINSIM_INB(cond, bit) ((cond) ? true : spinsim_bounds_fail(bit))
// Host side of the translation unit's word (read, then cleared when asked).
#define SPINSIM_BOUNDS_READER(name)                                                                       \
    uint64_t name(bool clear)                                                                             \
    {                                                                                                     \
        unsigned long long w = 0;                                                                         \
        if (cudaMemcpyFromSymbol(&w, g_spinsim_bounds_word, sizeof(w)) != cudaSuccess) return ~0ULL;     \
        if (clear) {                                                                                      \
            const unsigned long long z = 0;                                                               \
            if (cudaMemcpyToSymbol(g_spinsim_bounds_word, &z, sizeof(z)) != cudaSuccess) return ~0ULL;   \
        }                                                                                                 \
        return (uint64_t)w;                                                                               \
    }
#else
#define SPINSIM_INB(cond, bit) true
#endif
