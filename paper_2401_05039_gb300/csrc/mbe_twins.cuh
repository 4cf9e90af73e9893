// Twin classes of a frame's candidates, for the pruned kernel variants.
//
// iMBE's L - L' removal (Section II-C, embedded pruning): a candidate whose
// neighbourhood in L equals that of a candidate popped before it leaves P at
// that earlier pop (it could only lead to nodes that the earlier one, in Q
// from then on, rejects), and it joins neither P' nor Q'. The removal is
// applied whether or not the earlier candidate's own node is maximal, so
// the removed set is fixed when the frame is built and travels with it: a
// donated copy prunes exactly as its owner would. rep[j] = the first
// position whose row (its neighbourhood in L) equals row j, j itself when
// there is none.
//
// The classes come from one sort: every P row gets the key (digest, position)
// -- the digest is the row itself when |L| <= kTwinExactBits, else 24 bits
// of a hash of its words -- so equal rows end up next to each other in
// position order, and a row's representative is the first row of its group
// with the same words (compared word by word when the digest is a hash).
// The kernels sort with their own warp radix sort between twin_keys and
// twin_assign. pre[j] counts the removed positions before j (the byte
// count's |Q| at a pop).
#pragma once
#include <stdint.h>

namespace mbe {
namespace twins {
namespace { // one copy per kernel translation unit

constexpr unsigned kFullMask = 0xffffffffu;

// Word w of row k in 32-row tiles of W words (the layout of both kernels).
__device__ __forceinline__ int64_t tile_word(int k, int w, int W)
{
    return ((int64_t)(k >> 5) * W + w) * 32 + (k & 31);
}

__device__ __forceinline__ uint64_t row_digest(uint64_t h, uint64_t x)
{
    h ^= x + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2);
    return h * 0xbf58476d1ce4e5b9ULL;
}

constexpr int kTwinExactBits = 24; // level sets up to this size use the row itself as the digest

// Sort-key bits for n rows of a level set of m vertices.
__device__ __forceinline__ int twin_key_bits(int n, int m)
{
    const int pb = 32 - __clz(n > 1 ? n - 1 : 1);
    return (m < kTwinExactBits ? m : kTwinExactBits) + pb;
}

// keys[k] = (digest << pb) | k and vals[k] = k for the n rows at row indices
// off .. off + n - 1 of `rows` (W words each, m valid bits).
__device__ void twin_keys(int lane, const uint64_t *rows, int W, int off, int n, int m, uint64_t *keys,
                          int32_t *vals)
{
    const int pb = 32 - __clz(n > 1 ? n - 1 : 1);
    for (int k = lane; k < n; k += 32) {
        uint64_t d;
        if (m <= kTwinExactBits) {
            d = rows[tile_word(off + k, 0, W)]; // the row itself (bits >= m are zero)
        } else {
            uint64_t h = 0x9e3779b97f4a7c15ULL;
            for (int w = 0; w < W; ++w) h = row_digest(h, rows[tile_word(off + k, w, W)]);
            d = h >> (64 - kTwinExactBits);
        }
        keys[k] = (d << pb) | (uint64_t)k;
        vals[k] = k;
    }
    __syncwarp();
}

// rep[0..n) from the sorted keys / vals: the first position of each group of
// equal digests whose row equals the row (groups are in position order).
__device__ void twin_assign(int lane, const uint64_t *rows, int W, int off, int n, int m, const uint64_t *keys,
                            const int32_t *vals, int32_t *rep)
{
    const int pb = 32 - __clz(n > 1 ? n - 1 : 1);
    const bool exact = m <= kTwinExactBits;
    int carry = 0; // group start of the last entry of the previous chunk
    for (int base = 0; base < n; base += 32) {
        const int t = base + lane;
        const bool valid = t < n;
        const uint64_t g = valid ? keys[t] >> pb : ~0ULL;
        uint64_t gprev = __shfl_up_sync(kFullMask, g, 1);
        if (lane == 0) gprev = base > 0 ? keys[base - 1] >> pb : ~0ULL;
        const unsigned starts = __ballot_sync(kFullMask, valid && gprev != g);
        const unsigned upto = starts & (0xffffffffu >> (31 - lane)); // lanes <= lane
        const int gs = upto ? base + 31 - __clz(upto) : carry;
        if (valid) {
            const int p = vals[t];
            int r = p;
            if (exact) {
                r = vals[gs];
            } else {
                for (int h = gs; h < t; ++h) {
                    const int q = vals[h];
                    bool same = true;
                    for (int w = 0; w < W && same; ++w)
                        same = rows[tile_word(off + q, w, W)] == rows[tile_word(off + p, w, W)];
                    if (same) {
                        r = q;
                        break;
                    }
                }
            }
            rep[p] = r;
        }
        carry = __shfl_sync(kFullMask, gs, 31);
    }
    __syncwarp();
}

// Frames of at most 32 P rows (the common case): one lane per row, and
// equal rows found by one warp match on the row itself (W = 1) or on its
// digest, the digest match confirmed word by word. Returns false, having
// written nothing, when a digest matched rows that differ (then the sort
// path decides).
__device__ bool twin_small(int lane, const uint64_t *rows, int W, int off, int n, int32_t *rep, int32_t *pre)
{
    const bool valid = lane < n;
    uint64_t d = 0;
    if (valid) {
        if (W == 1) {
            d = rows[tile_word(off + lane, 0, 1)];
        } else {
            d = 0x9e3779b97f4a7c15ULL;
            for (int w = 0; w < W; ++w) d = row_digest(d, rows[tile_word(off + lane, w, W)]);
        }
    }
    const unsigned vm = __ballot_sync(kFullMask, valid);
    const unsigned grp = __match_any_sync(kFullMask, d) & vm;
    const int leader = valid ? __ffs(grp) - 1 : lane;
    bool ok = true;
    if (W > 1 && valid && leader != lane)
        for (int w = 0; w < W && ok; ++w)
            ok = rows[tile_word(off + leader, w, W)] == rows[tile_word(off + lane, w, W)];
    if (!__all_sync(kFullMask, ok)) return false;
    const unsigned rm = __ballot_sync(kFullMask, valid && leader < lane);
    if (valid) {
        rep[lane] = leader;
        pre[lane] = __popc(rm & ((1u << lane) - 1u));
    }
    __syncwarp();
    return true;
}

// The first position in [from, end) that is not removed (rep[k] == k), or
// end: removed candidates are passed over 32 at a time instead of one pop
// each.
__device__ __forceinline__ int next_kept(int lane, const int32_t *rep, int from, int end)
{
    for (int j = from; j < end; j += 32) {
        const int k = j + lane;
        const unsigned b = __ballot_sync(kFullMask, k < end && rep[k] == k);
        if (b) return j + __ffs(b) - 1;
    }
    return end;
}

// pre[j] = how many positions before j are removed (rep[k] < k), j < n.
__device__ void set_pre(int lane, const int32_t *rep, int n, int32_t *pre)
{
    int carry = 0;
    for (int base = 0; base < n; base += 32) {
        const int k = base + lane;
        const unsigned b = __ballot_sync(kFullMask, k < n && rep[k] < k);
        if (k < n) pre[k] = carry + __popc(b & ((1u << lane) - 1u));
        carry += __popc(b);
    }
    __syncwarp();
}

} // namespace
} // namespace twins
} // namespace mbe
