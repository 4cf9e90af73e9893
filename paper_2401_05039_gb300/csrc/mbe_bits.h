// Bit-level helpers shared by the search kernels and their host-side unit test.
// Plain C++ so that both nvcc (device) and g++ (host test) compile it.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define MBE_HD __host__ __device__ __forceinline__
#else
#define MBE_HD inline
#endif

namespace mbe {

// One SplitMix64 output step (Steele, Lea & Flood, OOPSLA 2014): add the
// golden gamma, then the variant-13 mix. Used for the order-independent
// biclique digest: key(u in U) = SM(2u), key(v in V) = SM(2v + 1).
MBE_HD uint64_t splitmix(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
MBE_HD uint64_t key_u(int32_t u) { return splitmix(2ULL * (uint64_t)(uint32_t)u); }
MBE_HD uint64_t key_v(int32_t v) { return splitmix(2ULL * (uint64_t)(uint32_t)v + 1ULL); }

// Bit compression ("generalized extract", Warren, Hacker's Delight 2nd ed.,
// Section 7-4): gather the bits of x selected by mask m into the low end,
// keeping their order. Every selected bit moves right by the number of
// unselected positions below it; that distance is applied in six stages of
// 1, 2, 4, 8, 16 and 32 positions, stage i moving the bits whose distance
// has bit i set. The six stage masks depend only on m, so a warp computes
// them once per level set and then compresses every candidate row with
// three operations per stage.
struct CompressMasks {
    uint64_t m;     // the selection mask itself
    uint64_t mv[6]; // bits that move at stage i (positions before that stage)
};

// Stage i of the mask preparation: the bits of m that move at this stage.
MBE_HD uint64_t compress_stage(uint64_t &m, uint64_t &zeros_below, int i)
{
    // prefix parity from the right of zeros_below: bit j is the parity of the
    // count of marked positions at or below j, i.e. bit i of each selected
    // bit's remaining move distance
    uint64_t par = zeros_below ^ (zeros_below << 1);
    par ^= par << 2;
    par ^= par << 4;
    par ^= par << 8;
    par ^= par << 16;
    par ^= par << 32;
    const uint64_t move = par & m;
    m = (m ^ move) | (move >> (1 << i));
    zeros_below &= ~par;
    return move;
}

MBE_HD CompressMasks compress_prepare(uint64_t m)
{
    CompressMasks c;
    c.m = m;
    uint64_t zeros_below = ~m << 1; // marks positions that have an unselected bit just below them
    for (int i = 0; i < 6; ++i) c.mv[i] = compress_stage(m, zeros_below, i);
    return c;
}

// The same masks with the six stages kept as a loop on the device (smaller
// code, for kernels whose hot loop must stay in the instruction cache).
MBE_HD CompressMasks compress_prepare_rolled(uint64_t m)
{
    CompressMasks c;
    c.m = m;
    uint64_t zeros_below = ~m << 1;
#if defined(__CUDA_ARCH__)
#pragma unroll 1
#endif
    for (int i = 0; i < 6; ++i) c.mv[i] = compress_stage(m, zeros_below, i);
    return c;
}

MBE_HD uint64_t compress_apply(uint64_t x, const CompressMasks &c)
{
    x &= c.m;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        uint64_t t = x & c.mv[i];
        x = (x ^ t) | (t >> (1 << i));
    }
    return x;
}

} // namespace mbe
