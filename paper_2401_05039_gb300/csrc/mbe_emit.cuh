// Biclique output of the search kernels (Algorithm 1's emit step when the
// caller asks for the bicliques themselves, not only count and hash).
//
// A biclique is written as one record |R|, |L|, R ids ascending, L ids
// ascending (global ids). Space is reserved with two atomic counters, one
// for ids and one for records; they keep counting past the caller's
// capacities, so at the end they hold the sizes the whole output needs.
// A record that does not fit is not written and raises the launch's
// output-full flag, which is separate from its error status: the search
// goes on, and count and hash stay exact.
//
// Both kernels keep the R of every frame in ascending order: a child's R is
// the merge of its parent's R with {x} and the candidates that joined R'
// at this node, sorted in scratch. L needs no sort: the level sets hold
// their vertices in ascending id order whenever output is requested.
#pragma once
#include <stdint.h>

#include "mbe_internal.h"

namespace mbe {
namespace emit {
namespace { // one copy per kernel translation unit

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Ascending sort of n distinct non-negative ids a[0..n) below 2^key_bits,
// with tmp[0..n) as the second buffer and hist (256 words of shared memory)
// for the digit counts. n <= 32: bitonic network in registers; larger: LSD
// radix sort over 8-bit digits, each pass a stable scatter ranked by
// __match_any_sync. Out of line: one copy for every call site.
__device__ __noinline__ void sort_ids(int lane, uint32_t *hist, int32_t *a, int32_t *tmp, int n, int key_bits)
{
    if (n <= 1) return;
    if (n <= 32) {
        int32_t v = lane < n ? a[lane] : 0x7fffffff;
#pragma unroll 1
        for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                const int32_t o = __shfl_xor_sync(kFull, v, stride);
                const bool up = (lane & size) == 0;
                const bool lower = (lane & stride) == 0;
                const bool want_min = lower == up;
                v = want_min ? min(v, o) : max(v, o);
            }
        }
        if (lane < n) a[lane] = v;
        __syncwarp();
        return;
    }
    const int passes = (key_bits + 7) / 8;
    int32_t *src = a, *dst = tmp;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        for (int b = lane; b < 256; b += 32) hist[b] = 0;
        __syncwarp();
        for (int k = lane; k < n; k += 32) atomicAdd(&hist[((uint32_t)src[k] >> shift) & 255u], 1u);
        __syncwarp();
        // exclusive scan of the 256 bins: lane l owns bins 8l .. 8l+7
        uint32_t loc[8], s = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            loc[j] = hist[8 * lane + j];
            s += loc[j];
        }
        uint32_t incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        uint32_t run = incl - s;
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            hist[8 * lane + j] = run;
            run += loc[j];
        }
        __syncwarp();
        for (int t0 = 0; t0 < n; t0 += 32) {
            const int k = t0 + lane;
            const bool valid = k < n;
            const int32_t v = valid ? src[k] : 0;
            const int d = valid ? (int)(((uint32_t)v >> shift) & 255u) : 256 + lane;
            const unsigned peers = __match_any_sync(kFull, d);
            const int rank = __popc(peers & lanemask_lt());
            const uint32_t base = valid ? hist[d] : 0;
            __syncwarp();
            if (valid) {
                dst[base + rank] = v;
                if (rank == 0) hist[d] = base + __popc(peers);
            }
            __syncwarp();
        }
        int32_t *t = src;
        src = dst;
        dst = t;
    }
    if (src != a) {
        for (int k = lane; k < n; k += 32) a[k] = src[k];
        __syncwarp();
    }
}

// Number of entries of the ascending list s[0..n) that are smaller than x.
__device__ __forceinline__ int rank_in(const int32_t *s, int n, int32_t x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// dst[0 .. na+nb) = merge of the ascending, disjoint lists A and B: every
// element lands at its own index plus its rank in the other list.
__device__ __forceinline__ void merge_into(int lane, const int32_t *A, int na, const int32_t *B, int nb, int32_t *dst)
{
    for (int k = lane; k < na; k += 32) {
        const int32_t x = A[k];
        dst[k + rank_in(B, nb, x)] = x;
    }
    for (int k = lane; k < nb; k += 32) {
        const int32_t x = B[k];
        dst[k + rank_in(A, na, x)] = x;
    }
    __syncwarp();
}

// Reserves one record of `need` ids. Returns the id offset of the record,
// or -1 when it does not fit (the output-full flag is then raised). Every
// lane gets the same answer.
__device__ __forceinline__ int64_t reserve(const SearchArgs &a, int lane, int64_t need, int64_t *rec)
{
    unsigned long long pos = 0, b = 0;
    if (lane == 0) {
        pos = atomicAdd(a.used_ids, (unsigned long long)need);
        b = atomicAdd(a.used_bic, 1ULL);
    }
    pos = __shfl_sync(kFull, pos, 0);
    b = __shfl_sync(kFull, b, 0);
    if ((int64_t)b >= a.cap_bic || (int64_t)(pos + need) > a.cap_ids) {
        if (lane == 0) atomicExch(a.out_full, 1);
        return -1;
    }
    *rec = (int64_t)b;
    return (int64_t)pos;
}

} // namespace
} // namespace emit
} // namespace mbe
