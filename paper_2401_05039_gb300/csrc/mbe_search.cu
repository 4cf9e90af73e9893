// Persistent warp-worker search kernel for maximal biclique enumeration.
//
// Each warp is an independent worker that runs Algorithm 1 (MBEA, paper
// Section II-B) depth first over one task at a time:
//  - a root task is one iteration of the top-level while loop: candidate r
//    with L = V, Q = the top-level candidates popped before r and P = those
//    after it, in the order (degree, id) (Section II-C, candidate
//    selection: ascending |N(v) n L|, which is the degree when L = V);
//  - a stolen task is a suffix of one frame's remaining candidates, split
//    off by a busy worker when another worker is idle (Section III-C's
//    work stealing, here without grid-wide synchronisation).
//
// Data layout (replaces the paper's compact arrays and lookup tables,
// Section III-B and III-D): a root builds its local universe, the rows
// bit(N(u) n N(r)) over the positions of N(r) for every u in N2(r). A
// frame with level set L (m vertices) keeps
//  - its candidates P as rows packed to L (bit j = adjacency to the j-th
//    vertex of L), 64-bit words, in tiles of 32 rows stored word-major so
//    lane k of a warp reads row 32t+k with coalesced loads;
//  - its check set X = Q followed by P (in pop order) transposed, as m
//    columns: column j is a bitset over the positions of X of the members
//    adjacent to the j-th vertex of L. When the i-th entry of P is popped,
//    Algorithm 1's Q is exactly the prefix of nQ + i positions, so "some q
//    in Q has N(q) >= L'" is an AND of the |L'| columns of L' over that
//    prefix (the paper's reverse scanning, Section III-D: iterate over L'
//    instead of Q), 64 candidates per word, stopping as soon as it is
//    empty, and Q' is the OR of the same columns over the same prefix.
// A child frame re-packs P' rows to L', compresses the chosen columns by
// the Q' mask (bit compression of mbe_bits.h) and appends its own P' to
// them by a warp bit-matrix transpose, so deep frames stay small.
// Expansion (Algorithm 1, step 4) is AND + popcount over the later P rows,
// one candidate per lane, with warp ballots and prefix sums for
// compaction.
//
// Frames live on a per-warp stack in device memory (an arena slice); the
// stack top is L1/L2 resident. P' is ordered by (|N(v) n L'|, id) once when
// its frame is pushed, which is the order in which Algorithm 1 pops it
// because the counts are fixed while L' is fixed.
#include "mbe_bits.h"
#include "mbe_emit.cuh"
#include "mbe_internal.h"
#include "mbe_twins.cuh"

// MBE_LIST_PATH = 1 builds the variant with the sorted-list path for level
// sets wider than the bitset limit (mbe_search_lists.cu); it is launched only
// for graphs with such roots. MBE_PRUNE = 1 builds the pruned variant
// (mbe_search_prune.cu: iMBE's L - L' removal, bitset level sets only). The
// out-of-line calls and extra state of either would cost the plain variant
// registers, hence separate translation units.
#ifndef MBE_LIST_PATH
#define MBE_LIST_PATH 0
#endif
#ifndef MBE_PRUNE
#define MBE_PRUNE 0
#endif
#if MBE_PRUNE
#define MBE_SEARCH_KERNEL search_prune_kernel
#define MBE_VARIANT_FIT search_prune_fit_shape
#define MBE_VARIANT_LAUNCH launch_search_prune
#elif MBE_LIST_PATH
#define MBE_SEARCH_KERNEL search_lists_kernel
#define MBE_VARIANT_FIT search_lists_fit_shape
#define MBE_VARIANT_LAUNCH launch_search_lists
#else
#define MBE_SEARCH_KERNEL search_kernel
#endif

namespace mbe {
namespace {

// The extended variants (list path, pruning) also carry the size filter.
constexpr bool kExt = MBE_LIST_PATH != 0 || MBE_PRUNE != 0;
// The pruned variant: every frame carries, per P entry, the first position
// of its twin class and the number of removed entries before it
// (mbe_twins.cuh).
constexpr bool kPrune = MBE_PRUNE != 0;
// Biclique output runs in the extended variants only (the host launches
// one of them when the bicliques are asked for): the plain kernels carry no
// output code in their node loop.
__device__ __forceinline__ bool emitting(const SearchArgs &a) { return kExt && a.emit; }

constexpr unsigned kFull = 0xffffffffu;
// per-warp shared memory (u32 units): hist[256] u32, off[32] i32, masks [32][7] u64,
// active-word masks lw[32] u64, active-word indices aw[32] i32
constexpr int kSmemWords = 256 + 32 + 32 * 7 * 2 + 32 * 2 + 32 + 34 * 2;
// Loads in flight are balanced against code size: the kernel's hot loop
// has to stay in the instruction cache (measured: fewer unrolled loads here
// and a rolled sorting network ran the column kernel 6-12% faster).
constexpr int kTiles = 2;      // 32-row tiles whose loads a lane keeps in flight together
constexpr int kUnionLoads = 4; // column words a lane keeps in flight while forming Q'
constexpr int kGather = 2;    // source words of a child row gathered before compression
constexpr int kCopyLoads = 1; // words a lane copies per step in q_copy_columns (a rarely taken path)
// a child's Q' columns are compressed when that leaves at most 1/4 of the words
constexpr int kCompressNum = 1, kCompressDen = 4;
// roots whose neighbours' degrees sum to at least this order L by degree class
constexpr int64_t kDegSortMin = 8192;



__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint64_t warp_sum64(uint64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ int64_t pad16(int64_t b) { return (b + 15) & ~(int64_t)15; }

struct __align__(16) FrameHdr {
    int32_t m;       // |L|: bits per P row and number of X columns
    int32_t W;       // 64-bit words per P row
    int32_t nQ;      // |Q|: inherited maximality-check candidates
    int32_t nP;      // candidates to pop, sorted by (count, id)
    int32_t i;       // next P position to pop
    int32_t end;     // one past the last P position this worker pops
    int32_t root;    // top-level candidate of this subtree (graph-local id)
    int32_t graph;   // graph of the subtree
    uint64_t Rsum;   // sum of key_u over R
    int32_t nR;      // |R| stored in the frame (emit mode), else 0
    int32_t QW;      // 64-bit words per X column
    int64_t bytes;   // size of the frame
    int64_t parent;  // offset of the parent frame from the arena base, -1 at the bottom
    int32_t qpos;    // X positions before P (>= nQ: positions of no Q member are zero in every column)
    int32_t copy_hint; // 1 when the last child built from this frame copied its columns uncompressed
    int32_t rn;      // |R| (exact when bicliques are written or a minimum |R| is set)
    int32_t pad_;
};
static_assert(sizeof(FrameHdr) == kFrameHdrBytes, "frame header size");

struct Frame {
    FrameHdr *h;
    int32_t *Lid;    // [m] vertex ids of L (V side)
    uint64_t *Q;     // [m][QW] columns over X = Q then P (nQ + nP positions)
    int32_t *gid;    // [nP] P candidate ids (U side)
    uint64_t *rows;  // [ceil(nP/32)][W][32] P rows
    int32_t *rep;    // pruned variant: [nP] first P position with the same row (mbe_twins.cuh)
    int32_t *pre;    // pruned variant: [nP] removed P positions before j (rep[k] < k, k < j)
    int32_t *R;      // [nR]
};

// Bytes of the pruned variant's twin sections (none in the other variants).
// A removed P position needs no mask of its own: its bits are left out of
// the frame's columns, which are only read over the prefix of popped
// positions, so it is in no Q' (its row, still in the frame, lets it join
// R' at its representative's pop).
__device__ __forceinline__ int64_t twin_bytes(int nP, int QW)
{
    return kPrune ? 2 * pad16(4LL * nP) : 0;
}

__device__ __forceinline__ int64_t frame_bytes(int m, int QW, int nP, int W, int nR)
{
    int64_t tiles = (nP + 31) >> 5;
    // every section is a multiple of 16 bytes: frames are copied with 16-byte accesses
    return kFrameHdrBytes + pad16(4LL * m) + pad16(8LL * m * QW) + pad16(4LL * nP) + 256LL * W * tiles +
           twin_bytes(nP, QW) + pad16(4LL * nR);
}

__device__ __forceinline__ Frame frame_at(char *p, int m, int QW, int nP, int W)
{
    Frame f;
    f.h = reinterpret_cast<FrameHdr *>(p);
    char *q = p + kFrameHdrBytes;
    f.Lid = reinterpret_cast<int32_t *>(q);
    q += pad16(4LL * m);
    f.Q = reinterpret_cast<uint64_t *>(q);
    q += pad16(8LL * m * QW);
    f.gid = reinterpret_cast<int32_t *>(q);
    q += pad16(4LL * nP);
    f.rows = reinterpret_cast<uint64_t *>(q);
    q += 256LL * W * ((nP + 31) >> 5);
    f.rep = nullptr;
    f.pre = nullptr;
    if (kPrune) {
        f.rep = reinterpret_cast<int32_t *>(q);
        q += pad16(4LL * nP);
        f.pre = reinterpret_cast<int32_t *>(q);
        q += pad16(4LL * nP);
    }
    f.R = reinterpret_cast<int32_t *>(q);
    return f;
}

__device__ __forceinline__ Frame frame_of(char *p)
{
    const FrameHdr *h = reinterpret_cast<const FrameHdr *>(p);
    return frame_at(p, h->m, h->QW, h->nP, h->W);
}

__device__ __forceinline__ int64_t row_word(int k, int w, int W)
{
    return ((int64_t)(k >> 5) * W + w) * 32 + (k & 31);
}

struct GView {
    const int32_t *u_off, *u_adj, *v_off, *v_adj;
    int32_t nU, nV;
};

__device__ __forceinline__ GView gview(const SearchArgs &a, int g)
{
    GraphDesc d = a.graphs[g];
    GView v;
    v.u_off = a.u_off + d.u_off_base;
    v.v_off = a.v_off + d.v_off_base;
    v.u_adj = a.u_adj + d.edge_base;
    v.v_adj = a.v_adj + d.edge_base;
    v.nU = d.nU;
    v.nV = d.nV;
    return v;
}

// Scratch region of a warp's arena (top end), reused by every node.
struct Scratch {
    int32_t *qsrc;  // root: universe positions of the earlier-ranked candidates
    int32_t *psrc;  // P' source positions
    uint64_t *pkey; // P' sort keys (count << key_shift | id)
    int32_t *psrc2;
    uint64_t *pkey2;
    int32_t *rtmp;  // ids that join R' (emit)
    int32_t *ugid;  // root universe: candidate ids
    int32_t *jlist; // positions (in L) of the bits of L'
    uint64_t *mq;   // Q' mask over the inherited Q (one word per 64 candidates)
    int32_t *offq;  // exclusive prefix of popcount(mq) per word
    uint64_t *cmq;  // compress stage masks of every mq word (6 per word)
    uint64_t *urows;// root universe rows
    int64_t ncap;   // capacity of the lists
    int64_t urow_words;
};

struct Ctx {
    int lane;
    int wid;
    char *arena;
    char *limit;  // frames must end at or below this address
    Scratch s;
    int32_t *mark;
    uint32_t *hist;   // shared [256]: radix-sort histogram
    int32_t *off;     // shared [32]: bit offset of each L' word's first selected bit
    uint64_t *cm;     // shared [32][7]: per word mask + 6 compress stage masks
    uint64_t *lw;     // shared [32]: the nonzero words of L', in order
    int32_t *aw;      // shared [32]: their word indices
    uint64_t *sbuf;   // shared [34]: staging of compressed Q column words
    int na;           // number of nonzero words of L'
    unsigned long long *dbg; // this worker's progress record (tracing runs only, else null)
    uint64_t cnt, hash, nodes, bytes; // current task (uniform across lanes)
    uint64_t t_cnt, t_hash, t_nodes, t_bytes, t_don, t_steal;
    int since_check;
    bool abort;
    uint64_t t_start; // globaltimer at kernel entry
    int depth;        // current stack depth (progress record)
};

// Progress record of a worker (debug builds of a run only).
__device__ __forceinline__ void trace(const SearchArgs &a, const Ctx &c, int phase, long long arg)
{
    if (c.dbg && c.lane == 0) {
        unsigned long long *d = c.dbg;
        d[0] = (unsigned long long)phase;
        d[1] = (unsigned long long)arg;
        d[2] = c.t_nodes + c.nodes;
        d[3] = (unsigned long long)c.depth;
        d[4] = c.t_don;
        d[5] = c.t_steal;
        d[6] = globaltimer() - c.t_start;
    }
}

// debug phase timer: ns since `since` added to bucket b (lane 0 only; no-op without tracing)
// MBE_TRACE = 1 compiles in the per-worker progress records and phase
// timers (mbe_debug_trace); off by default: the checks and timer reads cost
// the search 5-13% (measured on all five workloads).
#ifndef MBE_TRACE
#define MBE_TRACE 0
#endif
__device__ __forceinline__ uint64_t tnow(const SearchArgs &a)
{
    return (MBE_TRACE && a.debug) ? globaltimer() : 0;
}
__device__ __forceinline__ void tadd(const SearchArgs &a, Ctx &c, int b, uint64_t since)
{
    if (c.dbg) c.dbg[8 + b] += globaltimer() - since;
}

__device__ __forceinline__ bool past_deadline(const SearchArgs &a, const Ctx &c)
{
    return (long long)(globaltimer() - c.t_start) > a.deadline_ns;
}

__device__ __forceinline__ void set_error(const SearchArgs &a, int code)
{
    atomicCAS(a.error, 0, code);
}

// ------------------------------------------------------------------ sorting
// Ascending sort of n (key, value) pairs held in scratch; result in (k0, v0).
// n <= 32: bitonic network in registers; larger: LSD radix sort, 8-bit
// digits, stable scatter by warp ranking (match_any + popc).
// Kept out of line: one copy serves every call site, which keeps the
// kernel's hot loop small in the instruction cache.
__device__ __noinline__ void warp_sort_impl(int lane, uint32_t *hist_smem, uint64_t *k0, int32_t *v0, uint64_t *k1,
                                            int32_t *v1, int n, int key_bits)
{
    if (n <= 1) return;
    if (n <= 32) {
        uint64_t key = lane < n ? k0[lane] : ~0ULL;
        int32_t val = lane < n ? v0[lane] : 0;
#pragma unroll 1
        for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                uint64_t ok = __shfl_xor_sync(kFull, key, stride);
                int32_t ov = __shfl_xor_sync(kFull, val, stride);
                bool up = (lane & size) == 0;
                bool lower = (lane & stride) == 0;
                bool want_min = (lower == up);
                bool take = want_min ? (ok < key) : (ok > key);
                if (take) {
                    key = ok;
                    val = ov;
                }
            }
        }
        if (lane < n) {
            k0[lane] = key;
            v0[lane] = val;
        }
        __syncwarp();
        return;
    }
    int passes = (key_bits + 7) / 8;
    uint32_t *hist = hist_smem;
    for (int pass = 0; pass < passes; ++pass) {
        int shift = pass * 8;
        for (int b = lane; b < 256; b += 32) hist[b] = 0;
        __syncwarp();
        for (int t0 = 0; t0 < n; t0 += 32) {
            int k = t0 + lane;
            if (k < n) atomicAdd(&hist[(k0[k] >> shift) & 255], 1u);
        }
        __syncwarp();
        // exclusive scan of the 256 bins: lane l owns bins 8l..8l+7
        uint32_t loc[8], s = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            loc[j] = hist[lane * 8 + j];
            s += loc[j];
        }
        uint32_t incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        uint32_t run = incl - s;
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            hist[lane * 8 + j] = run;
            run += loc[j];
        }
        __syncwarp();
        for (int t0 = 0; t0 < n; t0 += 32) {
            int k = t0 + lane;
            bool valid = k < n;
            uint64_t key = valid ? k0[k] : 0;
            int32_t val = valid ? v0[k] : 0;
            int d = valid ? (int)((key >> shift) & 255) : 256 + lane;
            unsigned peers = __match_any_sync(kFull, d);
            int rank = __popc(peers & lanemask_lt());
            uint32_t base = valid ? hist[d] : 0;
            __syncwarp();
            if (valid) {
                k1[base + rank] = key;
                v1[base + rank] = val;
                if (rank == 0) hist[d] = base + __popc(peers);
            }
            __syncwarp();
        }
        uint64_t *tk = k0;
        k0 = k1;
        k1 = tk;
        int32_t *tv = v0;
        v0 = v1;
        v1 = tv;
    }
    if (passes & 1) { // result is in the second buffer: copy back
        for (int k = lane; k < n; k += 32) {
            k1[k] = k0[k];
            v1[k] = v0[k];
        }
        __syncwarp();
    }
}

__device__ __forceinline__ void warp_sort(Ctx &c, uint64_t *k0, int32_t *v0, uint64_t *k1, int32_t *v1, int n,
                                          int key_bits)
{
    warp_sort_impl(c.lane, c.hist, k0, v0, k1, v1, n, key_bits);
}

// Pruned variant: the twin sections (rep, pre) of a new frame whose n P
// rows (W words, m bits) are in place. Frames of at most 32 P rows take one
// warp match; larger ones (or a digest collision) one sort of (digest,
// position) keys. The sort lists are free again here (P' is in the frame).
// Out of line: it runs once per frame, and inlined it crowds the node
// loop out of the instruction cache (measured: Chung-Lu 20k 184 -> 160 ms).
__device__ __noinline__ void twin_sections(int lane, uint32_t *hist, const uint64_t *rows, int32_t *rep, int32_t *pre,
                                           uint64_t *k0, int32_t *v0, uint64_t *k1, int32_t *v1, int W, int off, int n,
                                           int m)
{
    if (n <= 32 && twins::twin_small(lane, rows, W, off, n, rep, pre)) return;
    twins::twin_keys(lane, rows, W, off, n, m, k0, v0);
    warp_sort_impl(lane, hist, k0, v0, k1, v1, n, twins::twin_key_bits(n, m));
    twins::twin_assign(lane, rows, W, off, n, m, k0, v0, rep);
    twins::set_pre(lane, rep, n, pre);
}

__device__ __forceinline__ void frame_twins(int lane, uint32_t *hist, const Scratch &S, const Frame &D, int W, int n,
                                            int m)
{
    twin_sections(lane, hist, D.rows, D.rep, D.pre, S.pkey2, S.psrc2, S.pkey, S.psrc, W, 0, n, m);
}

// ---------------------------------------------------------------- row scans
// Publishes the nonzero words of L' (lane w holds word w) as a compact list.
__device__ __forceinline__ void set_active_words(Ctx &c, uint64_t Lw)
{
    const unsigned act = __ballot_sync(kFull, Lw != 0);
    if (Lw != 0) {
        int pos = __popc(act & lanemask_lt());
        c.aw[pos] = c.lane;
        c.lw[pos] = Lw;
    }
    c.na = __popc(act);
    __syncwarp();
}

// cnt[u] = popcount(row & L') for row 32*(t0+u) + lane, u < T, over the
// nonzero words of L'. All loads of two words x T tiles are issued before
// they are consumed, so a lane keeps 2T independent loads in flight.
template <int T>
__device__ __forceinline__ void count_tiles(const Ctx &c, const uint64_t *rows, int W, int t0, int t_end,
                                            int (&cnt)[T])
{
#pragma unroll
    for (int u = 0; u < T; ++u) cnt[u] = 0;
    const uint64_t *base = rows + (int64_t)t0 * W * 32 + c.lane;
    const int64_t ts = (int64_t)W * 32;
    const int na = c.na;
    int wi = 0;
    for (; wi + 2 <= na; wi += 2) {
        const int w0 = c.aw[wi], w1 = c.aw[wi + 1];
        const uint64_t m0 = c.lw[wi], m1 = c.lw[wi + 1];
        uint64_t x0[T], x1[T];
#pragma unroll
        for (int u = 0; u < T; ++u) {
            const bool ok = t0 + u < t_end;
            x0[u] = ok ? base[u * ts + w0 * 32] : 0ULL;
            x1[u] = ok ? base[u * ts + w1 * 32] : 0ULL;
        }
#pragma unroll
        for (int u = 0; u < T; ++u) cnt[u] += __popcll(x0[u] & m0) + __popcll(x1[u] & m1);
    }
    if (wi < na) {
        const int w0 = c.aw[wi];
        const uint64_t m0 = c.lw[wi];
        uint64_t x0[T];
#pragma unroll
        for (int u = 0; u < T; ++u) x0[u] = (t0 + u < t_end) ? base[u * ts + w0 * 32] : 0ULL;
#pragma unroll
        for (int u = 0; u < T; ++u) cnt[u] += __popcll(x0[u] & m0);
    }
}

// ------------------------------------------------------------- child frames
// Lane w (< W) holds word w of L' in Lw. Publishes per-word compress masks
// and the bit offset of every word's first selected bit in shared memory.
__device__ __forceinline__ void prepare_offsets(Ctx &c, uint64_t Lw, int W)
{
    int pc = __popcll(Lw);
    int incl = pc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, incl, o);
        if (c.lane >= o) incl += y;
    }
    if (c.lane < W) c.off[c.lane] = incl - pc; // bit offset of word w
    __syncwarp();
}

__device__ __forceinline__ void prepare_cm(Ctx &c, uint64_t Lw, int W)
{
    if (c.lane < W) {
        CompressMasks cm = compress_prepare_rolled(Lw);
        uint64_t *dst = c.cm + c.lane * 7;
        dst[0] = Lw;
#pragma unroll
        for (int i = 0; i < 6; ++i) dst[1 + i] = cm.mv[i];
    }
    __syncwarp();
}

__device__ __forceinline__ void prepare_masks(Ctx &c, uint64_t Lw, int W)
{
    prepare_offsets(c, Lw, W);
    prepare_cm(c, Lw, W);
}

// Writes the rows of a child frame: row k' is source row src(k') of the
// source tile array, compressed to the bits of L' (masks from prepare_masks,
// active words from set_active_words). Source words are gathered kGather at a
// time before they are compressed.
__device__ void build_child_rows(Ctx &c, const uint64_t *srows, int Ws, const int32_t *psrc, int n,
                                 uint64_t *drows, int Wd)
{
    const int lane = c.lane;
    const int na = c.na;
    const int32_t *off = c.off;
    for (int t0 = 0; t0 < n; t0 += 32) {
        int k = t0 + lane;
        bool valid = k < n;
        int s = valid ? psrc[k] : 0;
        const uint64_t *src = srows + row_word(s, 0, Ws);
        uint64_t cur = 0;
        int o = 0;
        for (int wi = 0; wi < na; wi += kGather) {
            uint64_t x[kGather];
#pragma unroll
            for (int j = 0; j < kGather; ++j) x[j] = (valid && wi + j < na) ? src[c.aw[wi + j] * 32] : 0ULL;
#pragma unroll
            for (int j = 0; j < kGather; ++j) {
                if (wi + j >= na) break;
                const int w = c.aw[wi + j];
                const uint64_t *m = c.cm + w * 7;
                CompressMasks cm;
                cm.m = m[0];
#pragma unroll
                for (int q = 0; q < 6; ++q) cm.mv[q] = m[1 + q];
                uint64_t cw = compress_apply(x[j], cm);
                int bits = __popcll(cm.m);
                int b = off[w] & 63;
                cur |= cw << b;
                if (b + bits >= 64) {
                    drows[row_word(k, o, Wd)] = cur;
                    ++o;
                    cur = (b + bits > 64) ? (cw >> (64 - b)) : 0;
                }
            }
        }
        if (o < Wd) drows[row_word(k, o, Wd)] = cur;
    }
    __syncwarp();
}

// Compacts the ids of L at the positions J[0..m) (the bits of L') into dst.
__device__ __forceinline__ void compact_ids(Ctx &c, const int32_t *Lid, const int32_t *J, int m, int32_t *dst)
{
    for (int t = c.lane; t < m; t += 32) dst[t] = Lid[J[t]];
    __syncwarp();
}

// Sum of key_v over the ids of L at the positions J[0..m).
__device__ __forceinline__ uint64_t sum_keys_v(Ctx &c, const int32_t *Lid, const int32_t *J, int m)
{
    uint64_t s = 0;
    for (int t = c.lane; t < m; t += 32) s += key_v(Lid[J[t]]);
    return warp_sum64(s);
}

// Appends one biclique to the caller's output buffer: |R|, |L|, R ids, L ids,
// each side ascending. R' is the merge of the frame's R (ascending) with
// B[0..nB) (x and the candidates that joined R', sorted); L' is the ids of
// L at the positions J (ascending ids: L is kept in id order when emitting).
__device__ void emit_biclique(const SearchArgs &a, Ctx &c, const int32_t *Rbase, int nRbase, const int32_t *B,
                              int nB, const int32_t *Lid, const int32_t *J, int mL)
{
    const int nR = nRbase + nB;
    int64_t rec = 0;
    const int64_t pos = emit::reserve(a, c.lane, 2 + (int64_t)nR + mL, &rec);
    if (pos < 0) return;
    int32_t *o = a.out_ids + pos;
    if (c.lane == 0) {
        a.out_offsets[rec] = pos;
        o[0] = nR;
        o[1] = mL;
    }
    emit::merge_into(c.lane, Rbase, nRbase, B, nB, o + 2);
    compact_ids(c, Lid, J, mL, o + 2 + nR);
}

// ---------------------------------------------------------------- Q columns
// Position (0..63) of the r-th set bit (r < popcount(x)) of x: a binary
// search over halves, quarters, ... with popcounts (six steps, no loop).
__device__ __forceinline__ int select_bit(uint64_t x, int r)
{
    int pos = 0;
    int n = __popc((uint32_t)x);
    if (r >= n) { r -= n; x >>= 32; pos += 32; }
    n = __popc((uint32_t)x & 0xffffu);
    if (r >= n) { r -= n; x >>= 16; pos += 16; }
    n = __popc((uint32_t)x & 0xffu);
    if (r >= n) { r -= n; x >>= 8; pos += 8; }
    n = __popc((uint32_t)x & 0xfu);
    if (r >= n) { r -= n; x >>= 4; pos += 4; }
    n = __popc((uint32_t)x & 0x3u);
    if (r >= n) { r -= n; x >>= 2; pos += 2; }
    if (r >= (int)(x & 1u)) pos += 1;
    return pos;
}

// Positions (in L) of the mp bits of L', ascending (lane w holds word w of
// L'): lane t finds the t-th one directly (its active word by a binary
// search over the word offsets of prepare_offsets, then the bit by
// select_bit), so no lane walks many bits one by one. Needs
// set_active_words and prepare_offsets.
// An L' of at most kSerialBits bits is listed by each word's lane walking its
// bits (cheaper for a few bits); a longer one by the direct selection.
constexpr int kSerialBits = 8;

__device__ __forceinline__ void bit_positions(Ctx &c, uint64_t Lw, int W, int mp, int32_t *dst)
{
    if (mp <= kSerialBits) {
        if (c.lane < W) {
            int pos = c.off[c.lane];
            uint64_t b = Lw;
            while (b) {
                int t = __ffsll(b) - 1;
                b &= b - 1;
                dst[pos++] = c.lane * 64 + t;
            }
        }
        __syncwarp();
        return;
    }
    for (int t = c.lane; t < mp; t += 32) {
        int lo = 0, hi = c.na - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (c.off[c.aw[mid]] <= t) lo = mid;
            else hi = mid - 1;
        }
        const int w = c.aw[lo];
        dst[t] = w * 64 + select_bit(c.lw[lo], t - c.off[w]);
    }
    __syncwarp();
}

// True when some position p < lim of X has N(p) >= L': the AND of the
// columns listed in J (stride QW words), over the first LW = ceil(lim/64)
// words with the last one cut by `last`, is nonempty. Two columns of four
// words per lane in flight; a 128-word chunk stops as soon as its running
// AND is empty.
__device__ bool q_any_superset(const Ctx &c, const uint64_t *Q, int QW, int LW, uint64_t last, const int32_t *J,
                               int mp)
{
    const int lane = c.lane;
    for (int w0 = 0; w0 < LW; w0 += 128) {
        uint64_t acc[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int w = w0 + 32 * k + lane;
            acc[k] = w < LW ? (w == LW - 1 ? last : ~0ULL) : 0ULL;
        }
        for (int t = 0; t < mp; t += 2) {
            const bool two = t + 1 < mp;
            const uint64_t *col0 = Q + (int64_t)J[t] * QW + w0 + lane;
            const uint64_t *col1 = Q + (int64_t)J[two ? t + 1 : t] * QW + w0 + lane;
            uint64_t x[4], y[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool ok = w0 + 32 * k + lane < LW;
                x[k] = ok ? col0[32 * k] : 0ULL;
                y[k] = ok ? col1[32 * k] : 0ULL;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] &= x[k] & y[k];
            if (!__any_sync(kFull, (acc[0] | acc[1] | acc[2] | acc[3]) != 0)) break;
        }
        if (__any_sync(kFull, (acc[0] | acc[1] | acc[2] | acc[3]) != 0)) return true;
    }
    return false;
}

// Q' over the prefix of X: mq = OR of the columns listed in J (stride QW)
// over the first LW words, the last cut by `last`. Eight loads per lane in
// flight. Returns |Q'|.
__device__ int q_union(Ctx &c, const uint64_t *Q, int QW, int LW, uint64_t last, const int32_t *J, int mp)
{
    const int lane = c.lane;
    Scratch &S = c.s;
    int total = 0;
    for (int w0 = 0; w0 < LW; w0 += 32) {
        const int w = w0 + lane;
        const bool v = w < LW;
        const uint64_t *base = Q + (v ? w : 0);
        uint64_t m = 0;
        int jreg = 0;
        for (int t = 0; t < mp; t += kUnionLoads) {
            if ((t & 31) == 0) jreg = t + lane < mp ? J[t + lane] : 0;
            uint64_t x[kUnionLoads];
#pragma unroll
            for (int k = 0; k < kUnionLoads; ++k) {
                const int j = __shfl_sync(kFull, jreg, (t + k) & 31);
                x[k] = (v && t + k < mp) ? base[(int64_t)j * QW] : 0ULL;
            }
#pragma unroll
            for (int k = 0; k < kUnionLoads; ++k) m |= x[k];
        }
        if (w == LW - 1) m &= last;
        if (v) S.mq[w] = m;
        total += __popcll(m);
    }
    __syncwarp();
    return (int)__reduce_add_sync(kFull, (unsigned)total);
}

// q_union and, fused with it, the uncompressed child columns of
// q_copy_columns (every word loaded once, stored as it is OR-ed).
__device__ int q_union_copy(Ctx &c, const uint64_t *Q, int QW, int LW, uint64_t last, const int32_t *J, int mp,
                            uint64_t *dst, int QWd)
{
    const int lane = c.lane;
    Scratch &S = c.s;
    int total = 0;
    for (int w0 = 0; w0 < QWd; w0 += 32) {
        const int w = w0 + lane;
        const bool v = w < LW;
        const bool vd = w < QWd;
        const uint64_t cut = w == LW - 1 ? last : ~0ULL;
        const uint64_t *base = Q + (v ? w : 0);
        uint64_t m = 0;
        for (int t = 0; t < mp; t += kUnionLoads) {
            uint64_t x[kUnionLoads];
#pragma unroll
            for (int k = 0; k < kUnionLoads; ++k) {
                const int j = t + k < mp ? J[t + k] : 0;
                x[k] = (v && t + k < mp) ? (base[(int64_t)j * QW] & cut) : 0ULL;
            }
#pragma unroll
            for (int k = 0; k < kUnionLoads; ++k) {
                m |= x[k];
                if (vd && t + k < mp) dst[(int64_t)(t + k) * QWd + w] = x[k];
            }
        }
        if (v) S.mq[w] = m;
        total += __popcll(m);
    }
    __syncwarp();
    return (int)__reduce_add_sync(kFull, (unsigned)total);
}

// Compression of the prefix by mq: offq = per-word exclusive popcount
// prefix, cmq = compress stage masks of every word.
__device__ void q_compress_masks(int lane, const uint64_t *mq, int32_t *offq, uint64_t *cmq, int LW)
{
    int run = 0;
    for (int w0 = 0; w0 < LW; w0 += 32) {
        const int w = w0 + lane;
        const bool v = w < LW;
        const uint64_t m = v ? mq[w] : 0ULL;
        const int pc = __popcll(m);
        int incl = pc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        if (v) {
            offq[w] = run + incl - pc;
            CompressMasks cm = compress_prepare_rolled(m);
#pragma unroll
            for (int i = 0; i < 6; ++i) cmq[6 * (int64_t)w + i] = cm.mv[i];
        }
        run += __shfl_sync(kFull, incl, 31);
    }
    __syncwarp();
}

// Child column t = the first LW words of parent column J[t] (stride QW),
// last word cut by `last`, copied without compression: positions outside Q'
// are zero in every column of L' already. Words [LW, QWd) are zeroed for
// the P' bits that follow.
__device__ void q_copy_columns(int lane, const uint64_t *Q, int QW, int LW, uint64_t last, const int32_t *J, int mp,
                               uint64_t *dst, int QWd)
{
    // mp * QWd words: the frame fits the stack, far below 2^31 words
    const unsigned total = (unsigned)mp * (unsigned)QWd;
    for (unsigned b = 0; b < total; b += 32 * kCopyLoads) {
        uint64_t x[kCopyLoads];
        int64_t di[kCopyLoads];
#pragma unroll
        for (int u = 0; u < kCopyLoads; ++u) {
            const unsigned idx = b + 32 * u + lane;
            di[u] = -1;
            x[u] = 0;
            if (idx < total) {
                const int t = (int)(idx / (unsigned)QWd);
                const int w = (int)(idx - (unsigned)t * (unsigned)QWd);
                di[u] = idx;
                if (w < LW) {
                    x[u] = Q[(int64_t)J[t] * QW + w];
                    if (w == LW - 1) x[u] &= last;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kCopyLoads; ++u)
            if (di[u] >= 0) dst[di[u]] = x[u];
    }
    __syncwarp();
}

// Child column t = the first LW words of parent column J[t] (stride QW)
// compressed by mq, for every t < mp: each 32-word chunk of the parent
// column is compressed lane-wise and assembled in shared memory, then
// written out; only the first word of a chunk can hold bits of the previous
// chunk (it is OR-ed). dst is zeroed.
__device__ void q_child_columns(int lane, const uint64_t *mq, const uint64_t *cmq, const int32_t *offq, uint64_t *sbuf,
                                const uint64_t *Q, int QW, int LW, const int32_t *J, int mp, uint64_t *dst, int QWd)
{
    if (LW <= 8) {
        // short columns: one lane per child column, bits appended in registers
        for (int t = lane; t < mp; t += 32) {
            const uint64_t *col = Q + (int64_t)J[t] * QW;
            uint64_t *out = dst + (int64_t)t * QWd;
            uint64_t cur = 0;
            int o = 0, b = 0;
            for (int w = 0; w < LW; ++w) {
                CompressMasks cm;
                cm.m = mq[w];
#pragma unroll
                for (int i = 0; i < 6; ++i) cm.mv[i] = cmq[6 * (int64_t)w + i];
                const int nb = __popcll(cm.m);
                if (nb == 0) continue;
                const uint64_t v = compress_apply(col[w], cm);
                cur |= v << b;
                if (b + nb >= 64) {
                    out[o++] = cur;
                    cur = (b + nb > 64) ? (v >> (64 - b)) : 0;
                    b = b + nb - 64;
                } else {
                    b += nb;
                }
            }
            if (b > 0) out[o] = cur;
        }
        __syncwarp();
        return;
    }
    for (int t = 0; t < mp; ++t) {
        const uint64_t *col = Q + (int64_t)J[t] * QW;
        uint64_t *out = dst + (int64_t)t * QWd;
        for (int w0 = 0; w0 < LW; w0 += 32) {
            const int w = w0 + lane;
            const bool v = w < LW;
            uint64_t val = 0;
            int nb = 0, off = 0;
            if (v) {
                CompressMasks cm;
                cm.m = mq[w];
#pragma unroll
                for (int i = 0; i < 6; ++i) cm.mv[i] = cmq[6 * (int64_t)w + i];
                val = compress_apply(col[w], cm);
                nb = __popcll(cm.m);
                off = offq[w];
            }
            const int first = __shfl_sync(kFull, off, 0);
            const int k0 = first >> 6;
            const int last_lane = min(31, LW - 1 - w0);
            const int end_bit = __shfl_sync(kFull, off + nb, last_lane);
            if (end_bit == first) continue;
            const int k1 = (end_bit - 1) >> 6;
            for (int q = lane; q <= k1 - k0; q += 32) sbuf[q] = 0;
            __syncwarp();
            if (nb) {
                const int rel = off - (k0 << 6);
                const int kk = rel >> 6, b = rel & 63;
                atomicOr(reinterpret_cast<unsigned long long *>(&sbuf[kk]), (unsigned long long)(val << b));
                if (b + nb > 64)
                    atomicOr(reinterpret_cast<unsigned long long *>(&sbuf[kk + 1]),
                             (unsigned long long)(val >> (64 - b)));
            }
            __syncwarp();
            for (int q = lane; q <= k1 - k0; q += 32) out[k0 + q] = q == 0 ? (out[k0] | sbuf[0]) : sbuf[q];
            __syncwarp();
        }
    }
}

// Transpose of a 32 x 32 bit matrix held one row per lane (bit c of lane
// r's word = entry (r, c)): afterwards lane c holds column c (bit r = entry
// (r, c)). Recursive block transpose: at each of the five levels, lanes
// that differ in bit s swap the off-diagonal s x s blocks by one shuffle.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane)
{
    constexpr uint32_t kMask[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int s = 16 >> k;
        const uint32_t m = kMask[k];
        const uint32_t y = __shfl_xor_sync(kFull, x, s);
        x = (lane & s) ? ((x & ~m) | ((y >> s) & m)) : ((x & m) | ((y & m) << s));
    }
    return x;
}

// ORs 32 bits (rows t0..t0+31 of one column) into a column at bit p.
__device__ __forceinline__ void or_bits32(uint64_t *col, int p, uint32_t v)
{
    if (!v) return;
    uint64_t *cw = col + (p >> 6);
    const int b = p & 63;
    cw[0] |= (uint64_t)v << b;
    if (b > 32 && ((uint64_t)v >> (64 - b)) != 0) cw[1] |= (uint64_t)v >> (64 - b);
}

// Transposes n rows (tile layout, Wr words, row k taken from position
// pos[k] or k) into ncols column bitsets of QWd words, writing the rows as
// bits bit0 .. bit0+n-1 of every column (OR into zeroed columns). Each
// 32-row x 64-column block is two warp transposes. rep (pruned variant, or
// nullptr): row k is left out when rep[k] < k.
__device__ void rows_to_columns(int lane, const uint64_t *rows, int Wr, const int32_t *pos, int n, int ncols,
                                uint64_t *cols, int QWd, int bit0, const int32_t *rep = nullptr)
{
    for (int t0 = 0; t0 < n; t0 += 32) {
        const int k = t0 + lane;
        const bool valid = k < n && !(kPrune && rep && rep[k] < k);
        const int src = valid ? (pos ? pos[k] : k) : 0;
        const uint64_t *r = rows + row_word(src, 0, Wr);
        const int p = bit0 + t0;
        for (int w = 0; w * 64 < ncols; ++w) {
            const uint64_t x = valid ? r[w * 32] : 0ULL;
            const uint32_t lo = warp_transpose32((uint32_t)x, lane);
            const uint32_t hi = warp_transpose32((uint32_t)(x >> 32), lane);
            const int c0 = w * 64 + lane, c1 = c0 + 32;
            if (c0 < ncols) or_bits32(cols + (int64_t)c0 * QWd, p, lo);
            if (c1 < ncols) or_bits32(cols + (int64_t)c1 * QWd, p, hi);
        }
    }
    __syncwarp();
}

__device__ __forceinline__ void zero_words(Ctx &c, uint64_t *p, int64_t n)
{
    for (int64_t k = c.lane; k < n; k += 32) p[k] = 0;
    __syncwarp();
}

// ------------------------------------------------------------ node (frame)
// One iteration of Algorithm 1's while loop on the top frame at fp: pop
// x = P[i], build L' = L n N(x) (= row of x), check maximality against the
// inherited Q (column AND) and the P entries popped earlier (row scan),
// expand R' and collect P' from the later P entries, emit, and push the
// child frame when P' is nonempty. Returns the child's address or NULL.
__device__ char *process_node(const SearchArgs &a, Ctx &c, char *fp)
{
    const int lane = c.lane;
    Frame F = frame_of(fp);
    const int W = F.h->W, nQ = F.h->nQ, QW = F.h->QW, nP = F.h->nP;
    int i = F.h->i;
    if (kPrune && F.rep[i] < i) {
        // removed candidates are never popped (no node): go to the next one
        // still in P, or finish this worker's share of the frame
        const int end = F.h->end;
        i = twins::next_kept(lane, F.rep, i + 1, end);
        if (i >= end) {
            __syncwarp();
            if (lane == 0) F.h->i = end;
            return nullptr;
        }
    }
    __syncwarp(); // every lane has read the header before lane 0 advances the cursor
    if (lane == 0) F.h->i = i + 1;
    c.nodes += 1;

    // Step 2: L' = L n N(x) is the row of x (lane w holds word w).
    uint64_t t_scan = tnow(a);
    const uint64_t Lw = lane < W ? F.rows[row_word(i, lane, W)] : 0ULL;
    const int mp = __reduce_add_sync(kFull, (unsigned)__popcll(Lw));
    set_active_words(c, Lw);
    prepare_offsets(c, Lw, W);
    Scratch &S = c.s;
    int32_t *J = S.jlist;
    bit_positions(c, Lw, W, mp, J);

    // Step 3: maximality check against Algorithm 1's Q at this iteration:
    // the inherited Q and the P entries popped before x, i.e. the first
    // nQ + i positions of X (columns).
    const uint64_t t_q = tnow(a);
    const int lim = F.h->qpos + i;
    const int LW = (lim + 63) >> 6;
    const uint64_t last = (lim & 63) ? ((1ULL << (lim & 63)) - 1) : ~0ULL;
    const bool rejected = lim > 0 && q_any_superset(c, F.Q, QW, LW, last, J, mp);
    if (lane == 0) tadd(a, c, 14, t_q);
    if constexpr (kPrune) {
        // as below, with Q = the inherited Q and the P entries popped before
        // x (the removed ones are not); the later rows are added after the
        // expansion has counted the ones still in P
        const int nrm = F.pre[i];
        const uint64_t nq = (uint64_t)(nQ + i - nrm), rows = (uint64_t)W * nq, cols = (uint64_t)mp * ((nq + 63) >> 6);
        c.bytes += 8ULL * ((uint64_t)W + (rows < cols ? rows : cols));
    } else {
        // algorithmic bytes: x's row, the cheaper of the Q rows and the L'
        // columns over Q (|Q| = nQ + i here), and the later P rows when maximal
        const uint64_t nq = (uint64_t)(nQ + i), rows = (uint64_t)W * nq, cols = (uint64_t)mp * ((nq + 63) >> 6);
        c.bytes += 8ULL * ((uint64_t)W + (rows < cols ? rows : cols) + (rejected ? 0ULL : (uint64_t)W * (nP - i - 1)));
    }
    if (rejected) {
        if (lane == 0) tadd(a, c, 1, t_scan);
        return nullptr;
    }

    // Step 4: maximal expansion over P positions (i, nP).
    uint64_t rsum = 0;
    int pn = 0, nfull = 0, nrest = 0;
    const int ntiles = (nP + 31) >> 5;
    for (int t0 = (i + 1) >> 5; t0 < ntiles; t0 += kTiles) {
        int cnt[kTiles];
        count_tiles<kTiles>(c, F.rows, W, t0, ntiles, cnt);
#pragma unroll
        for (int u = 0; u < kTiles; ++u) {
            const int k = (t0 + u) * 32 + lane;
            bool valid = (t0 + u < ntiles) && k > i && k < nP;
            if (kPrune) {
                valid = valid && F.rep[k] >= i; // still in P at this pop
                nrest += __popc(__ballot_sync(kFull, valid));
            }
            const bool full = valid && cnt[u] == mp;
            const bool part = valid && cnt[u] > 0 && cnt[u] < mp && (!kExt || cnt[u] >= a.min_l);
            const int g = (full || part) ? F.gid[k] : 0;
            if (full) rsum += key_u(g);
            if (emitting(a) || (kExt && a.min_r > 1)) {
                const unsigned fb = __ballot_sync(kFull, full);
                if (emitting(a) && full) S.rtmp[nfull + __popc(fb & lanemask_lt())] = g;
                nfull += __popc(fb);
            }
            const unsigned bal = __ballot_sync(kFull, part);
            if (part) {
                const int p = pn + __popc(bal & lanemask_lt());
                S.pkey[p] = ((uint64_t)cnt[u] << a.key_shift) | (uint64_t)(uint32_t)g;
                S.psrc[p] = k;
            }
            pn += __popc(bal);
        }
    }
    if (lane == 0) tadd(a, c, 1, t_scan);
    if (kPrune) c.bytes += 8ULL * (uint64_t)W * (uint64_t)nrest;
    rsum = warp_sum64(rsum);
    const int xg = F.gid[i];
    const uint64_t Rs = F.h->Rsum + key_u(xg) + rsum;
    const uint64_t lsum = sum_keys_v(c, F.Lid, J, mp);
    // size filter (1, 1 by default: every biclique passes)
    const int rn = kExt ? F.h->rn + 1 + nfull : 0;
    const bool pass = !kExt || (rn >= a.min_r && mp >= a.min_l);
    if (pass) {
        c.cnt += 1;
        c.hash += splitmix(Rs + lsum);
    }

    uint64_t t_build = tnow(a);
    if (emitting(a)) {
        // B = {x} and the candidates that joined R', ascending
        if (lane == 0) S.rtmp[nfull] = xg;
        __syncwarp();
        emit::sort_ids(lane, c.hist, S.rtmp, S.psrc2, nfull + 1, a.key_shift);
        if (pass) emit_biclique(a, c, F.R, F.h->nR, S.rtmp, nfull + 1, F.Lid, J, mp);
    }
    // the child's level sets are smaller than L' and its R within R' u P'
    if (kExt && pn > 0 && (mp - 1 < a.min_l || rn + pn < a.min_r)) pn = 0;
    if (pn > 0) prepare_cm(c, Lw, W);
    if (pn == 0) {
        if (lane == 0) tadd(a, c, 2, t_build);
        return nullptr;
    }

    // Child frame: Q' (the members of the prefix touching L') as columns
    // over L', then P' rows sorted by (count, id), all packed to L'; the
    // child's X is Q' followed by P'. Q' is compressed to its members when
    // that shrinks the columns to at most kCompressNum/kCompressDen of the
    // prefix, else the prefix is copied with its holes.
    const int Wd = (mp + 63) >> 6;
    const int nRd = emitting(a) ? F.h->nR + 1 + nfull : 0;
    char *cp = fp + F.h->bytes;
    if ((uintptr_t)cp & 15) {
        if (lane == 0) set_error(a, kErrInternal);
        c.abort = true;
        return nullptr;
    }
    uint64_t t_qc = tnow(a);
    // When the previous child of this frame was copied, this one is copied
    // while Q' is formed (one pass over the words), before the choice.
    const int QWcopy = (lim + pn + 63) >> 6;
    const bool spec = lim > 0 && F.h->copy_hint != 0 && cp + frame_bytes(mp, QWcopy, pn, Wd, nRd) <= c.limit;
    uint64_t *dQ = reinterpret_cast<uint64_t *>(cp + kFrameHdrBytes + pad16(4LL * mp));
    int nQd = 0;
    if (spec)
        nQd = q_union_copy(c, F.Q, QW, LW, last, J, mp, dQ, QWcopy);
    else if (lim > 0)
        nQd = q_union(c, F.Q, QW, LW, last, J, mp);
    const bool compress = kCompressDen * ((nQd + 63) >> 6) <= kCompressNum * LW;
    if (lane == 0) F.h->copy_hint = compress ? 0 : 1;
    if (compress && nQd > 0) q_compress_masks(lane, S.mq, S.offq, S.cmq, LW);
    if (lane == 0) {
        tadd(a, c, 15, t_qc);
        tadd(a, c, 16, t_qc);
    }
    const int qposd = compress ? nQd : lim;
    const int QWd = (qposd + pn + 63) >> 6;
    const int64_t sz = frame_bytes(mp, QWd, pn, Wd, nRd);
    if (sz & 15) {
        if (lane == 0) set_error(a, kErrInternal);
        c.abort = true;
        return nullptr;
    }
    if (cp + sz > c.limit) {
        if (lane == 0) set_error(a, kErrArena);
        c.abort = true;
        return nullptr;
    }
    int key_bits = a.key_shift + (32 - __clz(mp));
    uint64_t t_sort = tnow(a);
    warp_sort(c, S.pkey, S.psrc, S.pkey2, S.psrc2, pn, key_bits);
    if (lane == 0 && c.dbg) {
        tadd(a, c, 4, t_sort);
        c.dbg[16] += nQd;
        c.dbg[17] += pn;
        c.dbg[18] += 1;
        c.dbg[19] += mp;
        c.dbg[20] += (uint64_t)W;
        c.dbg[21] += (uint64_t)(nQ + nP);
    }
    const uint64_t id_mask = (1ULL << a.key_shift) - 1;
    Frame D = frame_at(cp, mp, QWd, pn, Wd);
    for (int k = lane; k < pn; k += 32) D.gid[k] = (int32_t)(S.pkey[k] & id_mask);
    compact_ids(c, F.Lid, J, mp, D.Lid);
    build_child_rows(c, F.rows, W, S.psrc, pn, D.rows, Wd);
    if (kPrune) {
        const uint64_t t_tw = tnow(a);
        frame_twins(lane, c.hist, S, D, Wd, pn, mp);
        if (lane == 0) tadd(a, c, 22, t_tw);
    }
    t_qc = tnow(a);
    if (compress) {
        zero_words(c, D.Q, (int64_t)mp * QWd);
        if (nQd > 0) q_child_columns(lane, S.mq, S.cmq, S.offq, c.sbuf, F.Q, QW, LW, J, mp, D.Q, QWd);
    } else if (!spec) {
        q_copy_columns(lane, F.Q, QW, LW, last, J, mp, D.Q, QWd);
    }
    const uint64_t t_tr = tnow(a);
    rows_to_columns(lane, D.rows, Wd, nullptr, pn, mp, D.Q, QWd, qposd, D.rep);
    if (lane == 0 && c.dbg) {
        const uint64_t now = globaltimer();
        c.dbg[23] += now - t_qc;
        c.dbg[25] += t_tr - t_qc;
        c.dbg[26] += now - t_tr;
        c.dbg[27] += compress ? 0 : 1;
    }
    if (emitting(a)) emit::merge_into(lane, F.R, F.h->nR, S.rtmp, nfull + 1, D.R);
    if (lane == 0) {
        FrameHdr h;
        h.m = mp;
        h.W = Wd;
        h.nQ = nQd;
        h.nP = pn;
        h.i = 0;
        h.end = pn;
        h.root = F.h->root;
        h.graph = F.h->graph;
        h.Rsum = Rs;
        h.nR = nRd;
        h.QW = QWd;
        h.bytes = sz;
        h.parent = fp - c.arena;
        h.qpos = qposd;
        h.copy_hint = 1;
        h.rn = rn;
        h.pad_ = 0;
        *D.h = h;
        tadd(a, c, 2, t_build);
    }
    __syncwarp();
    return cp;
}

// ------------------------------------------------------ wide level sets
#include "mbe_list.cuh"

// A bitset child of a list node (mbe_list.cuh) in the column layout. One
// reverse scan over L' sets bit j of the universe row of every member of
// Q' u P' adjacent to L'[j]; the rows of P' are copied into the frame, and
// Q' and P' are transposed into its columns.
__device__ __noinline__ char *bits_from_lists(const SearchArgs &a, const ListEnv &e, char *cp, const GView &G,
                                              int graph, int root, int rn, int64_t parent, const int32_t *Lp,
                                              int mp, const int32_t *Qg, int nQd, const uint64_t *Pk, int pn,
                                              uint64_t Rs, const int32_t *Ra, int na, const int32_t *Rb, int nb)
{
    const int lane = e.lane;
    const int W = (mp + 63) >> 6, n = nQd + pn;
    const int64_t tiles = (n + 31) >> 5;
    const int QW = (n + 63) >> 6;
    const int nRd = emitting(a) ? na + nb : 0;
    const int64_t sz = frame_bytes(mp, QW, pn, W, nRd);
    if (n > e.ncap || tiles * W * 32 > e.urow_words || ((uintptr_t)cp & 15) || cp + sz > e.limit) {
        if (lane == 0) set_error(a, kErrArena);
        return nullptr;
    }
    const uint64_t id_mask = (1ULL << a.key_shift) - 1;
    for (int k = lane; k < n; k += 32) {
        const int u = k < nQd ? Qg[k] : (int32_t)(Pk[k - nQd] & id_mask);
        e.mark[u] = k;
        e.ugid[k] = u;
    }
    for (int64_t k = lane; k < tiles * W * 32; k += 32) e.urows[k] = 0;
    __syncwarp();
    uint64_t *urows = e.urows;
    reverse_scan(lane, G, Lp, mp, e.mark, [&](int k, int j) {
        atomicOr(reinterpret_cast<unsigned long long *>(&urows[row_word(k, j >> 6, W)]), 1ULL << (j & 63));
    });
    for (int k = lane; k < n; k += 32) e.mark[e.ugid[k]] = -1;
    Frame D = frame_at(cp, mp, QW, pn, W);
    for (int k = lane; k < pn; k += 32) D.gid[k] = e.ugid[nQd + k];
    for (int k = lane; k < mp; k += 32) D.Lid[k] = Lp[k];
    for (int64_t t = lane; t < (int64_t)pn * W; t += 32) {
        const int k = (int)(t / W), w = (int)(t - (int64_t)k * W);
        D.rows[row_word(k, w, W)] = urows[row_word(nQd + k, w, W)];
    }
    for (int64_t k = lane; k < (int64_t)mp * QW; k += 32) D.Q[k] = 0;
    __syncwarp();
    if (nQd > 0) rows_to_columns(lane, urows, W, nullptr, nQd, mp, D.Q, QW, 0);
    rows_to_columns(lane, D.rows, W, nullptr, pn, mp, D.Q, QW, nQd);
    if (emitting(a)) emit::merge_into(lane, Ra, na, Rb, nb, D.R);
    if (lane == 0) {
        FrameHdr h;
        h.m = mp;
        h.W = W;
        h.nQ = nQd;
        h.nP = pn;
        h.i = 0;
        h.end = pn;
        h.root = root;
        h.graph = graph;
        h.Rsum = Rs;
        h.nR = nRd;
        h.QW = QW;
        h.bytes = sz;
        h.parent = parent;
        h.qpos = nQd;
        h.copy_hint = 1;
        h.rn = rn;
        h.pad_ = 0;
        *D.h = h;
    }
    __syncwarp();
    return cp;
}

// The list path's view of a worker.
__device__ __forceinline__ ListEnv list_env(const Ctx &c)
{
    ListEnv e;
    e.lane = c.lane;
    e.mark = c.mark;
    e.hist = c.hist;
    e.arena = c.arena;
    e.limit = c.limit;
    e.qsrc = c.s.qsrc;
    e.psrc = c.s.psrc;
    e.psrc2 = c.s.psrc2;
    e.rtmp = c.s.rtmp;
    e.ugid = c.s.ugid;
    e.lbuf = reinterpret_cast<int32_t *>(c.s.urows + c.s.urow_words); // after the universe rows
    e.pkey = c.s.pkey;
    e.pkey2 = c.s.pkey2;
    e.urows = c.s.urows;
    e.ncap = c.s.ncap;
    e.urow_words = c.s.urow_words;
    return e;
}

__device__ __forceinline__ char *take_list_out(Ctx &c, const ListOut &o)
{
    c.cnt += o.cnt;
    c.hash += o.hash;
    c.bytes += o.bytes;
    if (o.abort) c.abort = true;
    return o.child;
}

// ------------------------------------------------------------- root task
// The top-level iteration for candidate r: L' = N(r), the root-local
// universe of N2(r), the check against the earlier-ranked candidates, the
// expansion by the later-ranked ones, and the level-1 frame at the bottom
// of the stack. Returns true when a frame was pushed.
constexpr bool kLists = MBE_LIST_PATH != 0 && MBE_PRUNE == 0;

__device__ bool process_root(const SearchArgs &a, Ctx &c, const GView &G, int r, int graph, int part, int parts)
{
    const int lane = c.lane;
    const uint64_t t_root = tnow(a);
    const int ro = G.u_off[r];
    const int d = G.u_off[r + 1] - ro;
    // never popped: an isolated vertex, one of degree below the size filter,
    // or (pruned variant) one with the neighbourhood of a smaller id: the
    // top-level L is V, so its twin class shares its degree and the smallest
    // id of the class is popped first
    if (d == 0 || (kExt && d < a.min_l)) return false;
    // (twin classes of this graph: local ids, indexed from its u_off base)
    const int32_t *trep = kPrune ? a.trep + a.graphs[graph].u_off_base : nullptr;
    if (kPrune && trep[r] < r) return false;
    // a pre-split root: every part rebuilds the root node, part 0 alone
    // counts it, and part p pops its own contiguous share of P'
    const bool first = part == 0;
    if (first) c.nodes += 1;
    const int W = (d + 63) >> 6;
    if (W > a.max_words) { // a sorted-list level set
        if constexpr (kLists) {
            return take_list_out(c, list_root(a, list_env(c), G, r, graph, part, parts)) != nullptr;
        } else {
            if (lane == 0) set_error(a, kErrInternal); // the host launches the list variant for such graphs
            c.abort = true;
            return false;
        }
    }
    Scratch &S = c.s;
    int32_t *mark = c.mark;

    // L = N(r) in ascending order of degree class (floor log2): column j of
    // every frame below is then about as sparse as the ones after it or
    // more, so the AND of a check meets its sparsest columns first and
    // empties early. Any order of L is valid (L is a set); it is applied
    // only when the root's candidate lists can be long (sum of the degrees
    // of N(r) at least kDegSortMin), and needs room in the lists.
    // (Not when the bicliques are written: they list L in id order, which the
    // level sets then keep.)
    const int32_t *Ln = G.u_adj + ro;
    if (!emitting(a) && d > 1 && d <= S.ncap) {
        int64_t sdeg = 0;
        for (int j = lane; j < d; j += 32) {
            const int w = G.u_adj[ro + j];
            const int dw = G.v_off[w + 1] - G.v_off[w];
            sdeg += dw;
            S.pkey[j] = ((uint64_t)min(31 - __clz(max(dw, 1)), 15) << 11) | (uint64_t)j;
            S.psrc[j] = w;
        }
        sdeg = (int64_t)warp_sum64((uint64_t)sdeg);
        __syncwarp();
        if (sdeg >= kDegSortMin) {
            warp_sort(c, S.pkey, S.psrc, S.pkey2, S.psrc2, d, 15);
            for (int j = lane; j < d; j += 32) S.jlist[j] = S.psrc[j];
            __syncwarp();
            Ln = S.jlist;
        }
    }

    // Discovery: for every (j, w = L[j]) and u in N(w), u != r, give u a
    // local id and set bit j of its row. Pairs are flattened across up to
    // 32 consecutive w so that lanes stay busy when degrees are small.
    int nc = 0, zeroed = 0;
    uint64_t pairs_total = 0;
    for (int j0 = 0; j0 < d; j0 += 32) {
        int j = j0 + lane;
        bool vj = j < d;
        int w = vj ? Ln[j] : 0;
        int wo = vj ? G.v_off[w] : 0;
        int wd = vj ? G.v_off[w + 1] - wo : 0;
        int incl = wd;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        const int excl = incl - wd;
        pairs_total += (uint64_t)total;
        for (int p0 = 0; p0 < total; p0 += 32) {
            int p = p0 + lane;
            bool vp = p < total;
            int s = 0; // last lane whose segment starts at or before p
#pragma unroll
            for (int b = 16; b > 0; b >>= 1) {
                int cand = s + b;
                int ex = __shfl_sync(kFull, excl, cand & 31);
                if (cand < 32 && ex <= p) s = cand;
            }
            int jj = j0 + s;
            int ws = __shfl_sync(kFull, wo, s);
            int es = __shfl_sync(kFull, excl, s);
            int u = vp ? G.v_adj[ws + (p - es)] : -1;
            bool take = vp && u != r;
            int cur = take ? mark[u] : 0;
            bool need = take && cur < 0;
            unsigned grp = __match_any_sync(kFull, need ? u : -2 - lane);
            int leader_lane = __ffs(grp) - 1;
            bool leader = need && leader_lane == lane;
            unsigned lb = __ballot_sync(kFull, leader);
            int newid = nc + __popc(lb & lanemask_lt());
            int nnew = __popc(lb);
            if (nc + nnew > S.ncap || (int64_t)((nc + nnew + 31) >> 5) * W * 32 > S.urow_words) {
                if (lane == 0) set_error(a, kErrArena);
                c.abort = true;
                break;
            }
            if (leader) {
                mark[u] = newid;
                S.ugid[newid] = u;
            }
            // zero every tile that gains its first row in this step
            while (zeroed * 32 < nc + nnew) {
                uint64_t *tile = S.urows + (int64_t)zeroed * W * 32;
                for (int q = lane; q < W * 32; q += 32) tile[q] = 0;
                ++zeroed;
            }
            nc += nnew;
            __syncwarp();
            int from = __shfl_sync(kFull, newid, leader_lane);
            int id = need ? from : cur;
            if (take) atomicOr(reinterpret_cast<unsigned long long *>(&S.urows[row_word(id, jj >> 6, W)]),
                               1ULL << (jj & 63));
        }
        if (c.abort) break;
    }
    __syncwarp();
    // reset the marks for the next root
    for (int k = lane; k < nc; k += 32) mark[S.ugid[k]] = -1;
    __syncwarp();
    if (first) c.bytes += 4ULL * ((uint64_t)d + pairs_total);
    if (c.abort) return false;

    // L' = N(r): all d bits (lane w holds word w)
    uint64_t Lw = 0;
    if (lane < W) Lw = (lane < W - 1 || (d & 63) == 0) ? ~0ULL : ((1ULL << (d & 63)) - 1);
    set_active_words(c, Lw);

    // Classify: earlier-ranked candidates (degree, id) < (d, r) form Q.
    uint64_t rsum = 0;
    int qn = 0, pn = 0, nfull = 0;
    const int utiles = (nc + 31) >> 5;
    for (int t0 = 0; t0 < nc; t0 += 32) {
        int k = t0 + lane;
        bool valid = k < nc;
        int cntv[1];
        count_tiles<1>(c, S.urows, W, t0 >> 5, utiles, cntv);
        int cnt = cntv[0], u = 0, du = 0;
        if (valid) {
            u = S.ugid[k];
            du = G.u_off[u + 1] - G.u_off[u];
        }
        // earlier-ranked candidates were popped before r (those below the size
        // filter never are); cnt > 0 for every discovered candidate
        const bool earlier = du < d || (du == d && u < r);
        // pruned: a later candidate left P at its twin's pop if that came
        // before r's; an earlier one that was removed never joined Q
        const bool removed = kPrune && valid && (earlier ? trep[u] < u : (du == d && trep[u] < r));
        bool ql = valid && !removed && earlier && (!kExt || du >= a.min_l);
        if (__ballot_sync(kFull, ql && cnt == d)) { // r's node is not maximal
            if (lane == 0) tadd(a, c, 0, t_root);
            return false;
        }
        bool full = valid && !removed && !earlier && cnt == d;
        bool qpart = ql;
        bool ppart = valid && !removed && !earlier && cnt < d && (!kExt || cnt >= a.min_l);
        if (full) rsum += key_u(u);
        if (emitting(a) || (kExt && a.min_r > 1)) {
            unsigned fb = __ballot_sync(kFull, full);
            if (emitting(a) && full) S.rtmp[nfull + __popc(fb & lanemask_lt())] = u;
            nfull += __popc(fb);
        }
        unsigned qb = __ballot_sync(kFull, qpart);
        if (qpart) S.qsrc[qn + __popc(qb & lanemask_lt())] = k;
        qn += __popc(qb);
        unsigned pb = __ballot_sync(kFull, ppart);
        if (ppart) {
            int p = pn + __popc(pb & lanemask_lt());
            S.pkey[p] = ((uint64_t)cnt << a.key_shift) | (uint64_t)(uint32_t)u;
            S.psrc[p] = k;
        }
        pn += __popc(pb);
    }
    rsum = warp_sum64(rsum);
    const uint64_t Rs = key_u(r) + rsum;
    uint64_t ls = 0;
    for (int j = lane; j < d; j += 32) ls += key_v(Ln[j]);
    ls = warp_sum64(ls);
    const bool pass = !kExt || 1 + nfull >= a.min_r; // d >= min_l already
    if (first && pass) {
        c.cnt += 1;
        c.hash += splitmix(Rs + ls);
    }

    prepare_masks(c, Lw, W);
    if (emitting(a)) {
        // R' = {r} and the candidates that joined it, ascending; L' = N(r)
        if (lane == 0) S.rtmp[nfull] = r;
        __syncwarp();
        emit::sort_ids(lane, c.hist, S.rtmp, S.psrc2, nfull + 1, a.key_shift);
        if (first && pass) {
            const int nR = 1 + nfull;
            int64_t rec = 0;
            const int64_t pos = emit::reserve(a, lane, 2 + (int64_t)nR + d, &rec);
            if (pos >= 0) {
                int32_t *o = a.out_ids + pos;
                if (lane == 0) {
                    a.out_offsets[rec] = pos;
                    o[0] = nR;
                    o[1] = d;
                }
                for (int k = lane; k < nR; k += 32) o[2 + k] = S.rtmp[k];
                for (int k = lane; k < d; k += 32) o[2 + nR + k] = Ln[k];
                __syncwarp();
            }
        }
    }
    if (pn == 0 || (kExt && (d - 1 < a.min_l || 1 + nfull + pn < a.min_r))) {
        if (lane == 0) tadd(a, c, 0, t_root);
        return false;
    }

    const int QW = (qn + pn + 63) >> 6;
    const int nRd = emitting(a) ? 1 + nfull : 0;
    const int64_t sz = frame_bytes(d, QW, pn, W, nRd);
    char *cp = c.arena;
    if (cp + sz > c.limit) {
        if (lane == 0) set_error(a, kErrArena);
        c.abort = true;
        return false;
    }
    int key_bits = a.key_shift + (32 - __clz(d));
    warp_sort(c, S.pkey, S.psrc, S.pkey2, S.psrc2, pn, key_bits);
    const uint64_t id_mask = (1ULL << a.key_shift) - 1;
    Frame D = frame_at(cp, d, QW, pn, W);
    for (int k = lane; k < pn; k += 32) D.gid[k] = (int32_t)(S.pkey[k] & id_mask);
    for (int k = lane; k < d; k += 32) D.Lid[k] = Ln[k];
    build_child_rows(c, S.urows, W, S.psrc, pn, D.rows, W);
    // X = the earlier-ranked candidates, then P in pop order, transposed
    // into one column per vertex of N(r)
    zero_words(c, D.Q, (int64_t)d * QW);
    if (qn > 0) rows_to_columns(lane, S.urows, W, S.qsrc, qn, d, D.Q, QW, 0);
    if (kPrune) {
        const uint64_t t_tw = tnow(a);
        frame_twins(lane, c.hist, S, D, W, pn, d);
        if (lane == 0) tadd(a, c, 22, t_tw);
    }
    rows_to_columns(lane, D.rows, W, nullptr, pn, d, D.Q, QW, qn, D.rep);
    if (emitting(a))
        for (int k = lane; k <= nfull; k += 32) D.R[k] = S.rtmp[k];
    if (lane == 0) {
        FrameHdr h;
        h.m = d;
        h.W = W;
        h.nQ = qn;
        h.nP = pn;
        h.i = (int32_t)(((int64_t)pn * part) / parts);
        h.end = (int32_t)(((int64_t)pn * (part + 1)) / parts);
        h.root = r;
        h.graph = graph;
        h.Rsum = Rs;
        h.nR = nRd;
        h.QW = QW;
        h.bytes = sz;
        h.parent = -1;
        h.qpos = qn;
        h.copy_hint = 1;
        h.rn = 1 + nfull;
        h.pad_ = 0;
        *D.h = h;
        tadd(a, c, 0, t_root);
    }
    __syncwarp();
    return true;
}

// ---------------------------------------------------------------- stealing
enum : int32_t { kSlotEmpty = 0, kSlotWriting = 1, kSlotFull = 2, kSlotTaken = 3 };

__device__ bool warp_copy(char *dst, const char *src, int64_t bytes, int lane, bool from_other_sm)
{
    // frames are 16-byte aligned multiples of 16 bytes; anything else is a bug: copy nothing
    if ((((uintptr_t)dst | (uintptr_t)src) & 15) || (bytes & 15) || bytes < 0) return false;
    const int4 *s = reinterpret_cast<const int4 *>(src);
    int4 *d = reinterpret_cast<int4 *>(dst);
    int64_t n = bytes >> 4;
    int64_t k = lane;
    for (; k + 96 < n; k += 128) {
        int4 v0, v1, v2, v3;
        if (from_other_sm) {
            v0 = __ldcg(s + k);
            v1 = __ldcg(s + k + 32);
            v2 = __ldcg(s + k + 64);
            v3 = __ldcg(s + k + 96);
        } else {
            v0 = s[k];
            v1 = s[k + 32];
            v2 = s[k + 64];
            v3 = s[k + 96];
        }
        d[k] = v0;
        d[k + 32] = v1;
        d[k + 64] = v2;
        d[k + 96] = v3;
    }
    for (; k < n; k += 32) d[k] = from_other_sm ? __ldcg(s + k) : s[k];
    __syncwarp();
    return true;
}

// The frame walk and copy of a donation: 1 when a frame was published, -1
// when the copy failed (the run aborts), 0 when no frame qualified. Out of
// line: it runs rarely, and the node loop keeps its instruction-cache room
// (measured: planted 5k 37.9 -> 35.3 ms, Chung-Lu 200k 477 -> 452 ms).
__device__ __noinline__ int donate_frame(const SearchArgs &a, int lane, int wid, char *arena, char *top)
{
    // walk frames from the bottom of the stack
    char *fp = arena;
    while (true) {
        FrameHdr *h = reinterpret_cast<FrameHdr *>(fp);
        int left = h->end - h->i;
        if (left >= 2 && h->bytes <= a.slot_bytes && h->bytes <= a.stack_bytes) {
            int mid = h->i + (left + 1) / 2;
            char *slot = a.slots + (int64_t)wid * a.slot_bytes;
            if (lane == 0) {
                a.slot_state[wid] = kSlotWriting;
                atomicAdd(reinterpret_cast<unsigned long long *>(a.outstanding), 1ULL);
            }
            __syncwarp();
            if (!warp_copy(slot, fp, h->bytes, lane, false)) {
                if (lane == 0) {
                    set_error(a, kErrInternal);
                    atomicExch(a.slot_state + wid, kSlotEmpty);
                    atomicAdd(reinterpret_cast<unsigned long long *>(a.outstanding), ~0ULL);
                }
                return -1;
            }
            if (lane == 0) {
                FrameHdr *sh = reinterpret_cast<FrameHdr *>(slot);
                sh->i = mid;
                sh->parent = -1;
                h->end = mid;
                __threadfence();
                atomicExch(a.slot_state + wid, kSlotFull);
                atomicAdd(a.n_published, 1);
            }
            __syncwarp();
            return 1;
        }
        if (fp == top) return 0;
        fp += h->bytes;
    }
}

// If some worker is idle and this worker's slot is free, give away the upper
// half of the remaining candidates of its shallowest frame that has at least
// two left: the copy keeps every candidate (earlier positions stay Q-like
// for the thief), with i = mid; this worker keeps [i, mid).
__device__ __forceinline__ void maybe_donate(const SearchArgs &a, Ctx &c, char *top)
{
    const int lane = c.lane;
    int idle = 0, state = 0;
    if (lane == 0) {
        idle = *reinterpret_cast<volatile int32_t *>(a.n_idle) -
               *reinterpret_cast<volatile int32_t *>(a.n_published);
        state = *reinterpret_cast<volatile int32_t *>(a.slot_state + c.wid);
    }
    idle = __shfl_sync(kFull, idle, 0);
    state = __shfl_sync(kFull, state, 0);
    if (idle <= 0 || state != kSlotEmpty) return;
    const uint64_t t_cp = tnow(a);
    const int r = donate_frame(a, lane, c.wid, c.arena, top);
    if (r < 0) c.abort = true;
    if (r > 0) {
        c.t_don += 1;
        if (lane == 0) tadd(a, c, 3, t_cp);
    }
}

// Claims a published frame: the own slot first, then the others circularly.
__device__ bool try_steal(const SearchArgs &a, Ctx &c)
{
    const int lane = c.lane;
    int pub = 0;
    if (lane == 0) pub = *reinterpret_cast<volatile int32_t *>(a.n_published);
    pub = __shfl_sync(kFull, pub, 0);
    if (pub <= 0) return false;
    const int nw = a.n_warps;
    for (int base = 0; base < nw; base += 32) {
        int idx = base + lane;
        int s = (c.wid + idx) % nw;
        int st = idx < nw ? *reinterpret_cast<volatile int32_t *>(a.slot_state + s) : kSlotEmpty;
        unsigned cand = __ballot_sync(kFull, st == kSlotFull);
        while (cand) {
            int l = __ffs(cand) - 1;
            cand &= cand - 1;
            int victim = (c.wid + base + l) % nw;
            int ok = 0;
            if (lane == 0) {
                ok = atomicCAS(a.slot_state + victim, kSlotFull, kSlotTaken) == kSlotFull;
                if (ok) atomicSub(a.n_published, 1);
            }
            ok = __shfl_sync(kFull, ok, 0);
            if (!ok) continue;
            __threadfence();
            const char *slot = a.slots + (int64_t)victim * a.slot_bytes;
            int64_t bytes = 0;
            if (lane == 0) bytes = __ldcg(reinterpret_cast<const long long *>(slot + 48));
            bytes = __shfl_sync(kFull, bytes, 0);
            if (bytes > a.stack_bytes || bytes > a.slot_bytes || bytes < 64) {
                // cannot happen for frames published by maybe_donate; refuse rather than overrun
                if (lane == 0) {
                    set_error(a, kErrArena);
                    atomicExch(a.slot_state + victim, kSlotEmpty);
                }
                c.abort = true;
                return false;
            }
            uint64_t t_cp = tnow(a);
            if (!warp_copy(c.arena, slot, bytes, lane, true)) {
                if (lane == 0) {
                    set_error(a, kErrInternal);
                    atomicExch(a.slot_state + victim, kSlotEmpty);
                }
                c.abort = true;
                return false;
            }
            if (lane == 0) tadd(a, c, 3, t_cp);
            __threadfence();
            if (lane == 0) atomicExch(a.slot_state + victim, kSlotEmpty);
            __syncwarp();
            if (victim != c.wid) c.t_steal += 1;
            return true;
        }
    }
    return false;
}

// Runs the frames on the stack until it is empty (or the run aborts).
__device__ void run_stack(const SearchArgs &a, Ctx &c, char *top)
{
    const int lane = c.lane;
    while (top != nullptr && !c.abort) {
        FrameHdr *h = reinterpret_cast<FrameHdr *>(top);
        if (h->i >= h->end) {
            int64_t par = h->parent;
            top = par < 0 ? nullptr : c.arena + par;
            c.depth -= 1;
            continue;
        }
        if (++c.since_check >= 16) {
            c.since_check = 0;
            int err = 0;
            if (lane == 0) {
                err = *reinterpret_cast<volatile int32_t *>(a.error);
                if (!err && past_deadline(a, c)) {
                    set_error(a, kErrTimeout);
                    err = kErrTimeout;
                }
            }
            err = __shfl_sync(kFull, err, 0);
            trace(a, c, 2, c.depth);
            if (err) {
                c.abort = true;
                break;
            }
            if (a.steal) maybe_donate(a, c, top);
        }
        char *child;
        if constexpr (kLists) {
            if (is_list_frame(top)) {
                c.nodes += 1;
                child = take_list_out(c, list_node(a, list_env(c), top));
            } else {
                child = process_node(a, c, top);
            }
        } else {
            child = process_node(a, c, top);
        }
        __syncwarp(); // header updates by lane 0 are visible to the whole warp
        if (child) {
            top = child;
            c.depth += 1;
        }
    }
    __syncwarp();
}

__device__ void finish_task(const SearchArgs &a, Ctx &c, int owner)
{
    if (c.lane == 0) {
        if (a.per_task_owner && owner >= 0) {
            unsigned long long *p = a.per_task_owner + 4LL * owner;
            atomicAdd(p + 0, (unsigned long long)c.cnt);
            atomicAdd(p + 1, (unsigned long long)c.hash);
            atomicAdd(p + 2, (unsigned long long)c.nodes);
            atomicAdd(p + 3, (unsigned long long)c.bytes);
        }
        atomicAdd(reinterpret_cast<unsigned long long *>(a.outstanding), ~0ULL); // -1
    }
    c.t_cnt += c.cnt;
    c.t_hash += c.hash;
    c.t_nodes += c.nodes;
    c.t_bytes += c.bytes;
    c.cnt = c.hash = c.nodes = c.bytes = 0;
    __syncwarp();
}

#ifndef MBE_SEARCH_MIN_BLOCKS
#define MBE_SEARCH_MIN_BLOCKS 2 // resident 256-thread blocks per SM the register budget is sized for
#endif
__global__ void __launch_bounds__(256, MBE_SEARCH_MIN_BLOCKS) MBE_SEARCH_KERNEL(const __grid_constant__ SearchArgs a)
{
    extern __shared__ uint32_t smem[];
    Ctx c;
    c.lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    c.wid = blockIdx.x * (blockDim.x >> 5) + wib;
    if (c.wid >= a.n_warps) return;
    uint32_t *my = smem + wib * kSmemWords;
    c.hist = my;
    c.off = reinterpret_cast<int32_t *>(my + 256);
    c.cm = reinterpret_cast<uint64_t *>(my + 256 + 32);
    c.lw = reinterpret_cast<uint64_t *>(my + 256 + 32 + 32 * 7 * 2);
    c.aw = reinterpret_cast<int32_t *>(my + 256 + 32 + 32 * 7 * 2 + 64);
    c.sbuf = reinterpret_cast<uint64_t *>(my + 256 + 32 + 32 * 7 * 2 + 64 + 32);
    c.na = 0;
    c.dbg = (MBE_TRACE && a.debug) ? a.debug + (int64_t)MBE_TRACE_WORDS * c.wid : nullptr;
    c.arena = a.arena + (int64_t)c.wid * a.arena_bytes;
    c.mark = a.mark + (int64_t)c.wid * a.mark_stride;
    {
        // scratch (top of the arena): seven candidate lists of n_cand_cap
        // entries, then the root universe rows
        char *q = c.arena + a.arena_bytes - a.scratch_bytes;
        c.limit = c.arena + a.stack_bytes;
        const int64_t nc = a.n_cand_cap;
        c.s.ncap = nc;
        c.s.qsrc = reinterpret_cast<int32_t *>(q);
        q += pad16(4 * nc);
        c.s.psrc = reinterpret_cast<int32_t *>(q);
        q += pad16(4 * nc);
        c.s.psrc2 = reinterpret_cast<int32_t *>(q);
        q += pad16(4 * nc);
        c.s.rtmp = reinterpret_cast<int32_t *>(q);
        q += pad16(4 * nc);
        c.s.ugid = reinterpret_cast<int32_t *>(q);
        q += pad16(4 * nc);
        c.s.pkey = reinterpret_cast<uint64_t *>(q);
        q += pad16(8 * nc);
        c.s.pkey2 = reinterpret_cast<uint64_t *>(q);
        q += pad16(8 * nc);
        const int64_t qw = (nc + 63) / 64 + 1;
        c.s.jlist = reinterpret_cast<int32_t *>(q);
        q += pad16(4 * 2048);
        c.s.mq = reinterpret_cast<uint64_t *>(q);
        q += pad16(8 * qw);
        c.s.offq = reinterpret_cast<int32_t *>(q);
        q += pad16(4 * qw);
        c.s.cmq = reinterpret_cast<uint64_t *>(q);
        q += pad16(56 * qw);
        c.s.urows = reinterpret_cast<uint64_t *>(q);
        c.s.urow_words = a.urow_bytes / 8;
    }
    c.cnt = c.hash = c.nodes = c.bytes = 0;
    c.t_cnt = c.t_hash = c.t_nodes = c.t_bytes = c.t_don = c.t_steal = 0;
    c.since_check = 0;
    c.abort = false;
    c.t_start = __shfl_sync(kFull, globaltimer(), 0);
    c.depth = 0;

    bool idle = false;
    uint64_t idle_since = 0;
    unsigned backoff = 64;
    while (true) {
        // 1) next root task in execution order
        long long t = -1;
        if (c.lane == 0) {
            if (*reinterpret_cast<volatile int32_t *>(a.error) == 0 &&
                (long long)*reinterpret_cast<volatile unsigned long long *>(a.cursor) < a.n_tasks) {
                atomicAdd(reinterpret_cast<unsigned long long *>(a.outstanding), 1ULL);
                t = (long long)atomicAdd(a.cursor, 1ULL);
                if (t >= a.n_tasks) {
                    atomicAdd(reinterpret_cast<unsigned long long *>(a.outstanding), ~0ULL);
                    t = -1;
                }
            }
        }
        t = __shfl_sync(kFull, t, 0);
        if (t >= 0) {
            if (idle && c.lane == 0) {
                atomicSub(a.n_idle, 1);
                if (c.dbg) c.dbg[29] += globaltimer() - idle_since; // idle between tasks
            }
            idle = false;
            int g = a.task_graph ? a.task_graph[t] : 0;
            int r = a.task_root[t];
            int sp = a.task_split ? a.task_split[t] : 0;
            int parts = sp ? (sp >> 16) : 1, part = sp ? (sp & 0xffff) : 0;
            GView G = gview(a, g);
            trace(a, c, 1, r);
            backoff = 64;
            uint64_t t_busy = tnow(a);
            bool pushed = process_root(a, c, G, r, g, part, parts);
            c.depth = pushed ? 1 : 0;
            if (pushed && !c.abort) run_stack(a, c, c.arena);
            if (c.lane == 0) {
                tadd(a, c, 5, t_busy);
                if (c.dbg) c.dbg[14] += 1;
            }
            finish_task(a, c, a.per_root_mode == 2 ? g : r);
            if (c.lane == 0 && c.dbg) c.dbg[28] = globaltimer() - c.t_start; // end of the last task
            if (c.abort) break;
            continue;
        }
        // 2) a published frame (own slot first)
        if (a.steal && try_steal(a, c)) {
            if (idle && c.lane == 0) {
                atomicSub(a.n_idle, 1);
                if (c.dbg) c.dbg[29] += globaltimer() - idle_since; // idle between tasks
            }
            idle = false;
            const FrameHdr *h = reinterpret_cast<const FrameHdr *>(c.arena);
            int owner = a.per_root_mode == 2 ? h->graph : h->root;
            trace(a, c, 3, owner);
            backoff = 64;
            c.depth = 1;
            uint64_t t_busy = tnow(a);
            run_stack(a, c, c.arena);
            if (c.lane == 0) {
                tadd(a, c, 5, t_busy);
                if (c.dbg) c.dbg[15] += 1;
            }
            finish_task(a, c, owner);
            if (c.lane == 0 && c.dbg) c.dbg[28] = globaltimer() - c.t_start; // end of the last task
            if (c.abort) break;
            continue;
        }
        // 3) idle: wait for work or for the end
        if (!idle) {
            if (c.lane == 0) atomicAdd(a.n_idle, 1);
            idle = true;
            idle_since = __shfl_sync(kFull, globaltimer(), 0);
        }
        int done = 0, err = 0;
        if (c.lane == 0) {
            long long out = *reinterpret_cast<volatile long long *>(a.outstanding);
            unsigned long long cur = *reinterpret_cast<volatile unsigned long long *>(a.cursor);
            done = (out == 0 && (long long)cur >= a.n_tasks);
            err = *reinterpret_cast<volatile int32_t *>(a.error);
        }
        done = __shfl_sync(kFull, done, 0);
        err = __shfl_sync(kFull, err, 0);
        if (done || err) {
            if (c.lane == 0) atomicSub(a.n_idle, 1);
            break;
        }
        // time-based decisions are taken by lane 0 and broadcast: each lane
        // reads its own timer, and lanes must never leave the loop apart
        int expired = 0;
        if (c.lane == 0) expired = (long long)(globaltimer() - idle_since) > a.watchdog_ns || past_deadline(a, c);
        expired = __shfl_sync(kFull, expired, 0);
        if (expired) {
            if (c.lane == 0) {
                set_error(a, kErrTimeout);
                atomicSub(a.n_idle, 1);
            }
            trace(a, c, 5, 0);
            break;
        }
        trace(a, c, 4, 0);
        __nanosleep(backoff);
        if (backoff < 8192) backoff <<= 1;
    }
    trace(a, c, 6, c.abort ? 1 : 0);
    if (c.lane == 0) {
        atomicAdd(a.totals + 0, (unsigned long long)c.t_cnt);
        atomicAdd(a.totals + 1, (unsigned long long)c.t_hash);
        atomicAdd(a.totals + 2, (unsigned long long)c.t_nodes);
        atomicAdd(a.totals + 3, (unsigned long long)c.t_bytes);
        atomicAdd(a.totals + 4, (unsigned long long)c.t_don);
        atomicAdd(a.totals + 5, (unsigned long long)c.t_steal);
    }
}

} // namespace

#if MBE_LIST_PATH || MBE_PRUNE

int MBE_VARIANT_FIT(int threads, int blocks_per_sm_req)
{
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, MBE_SEARCH_KERNEL) != cudaSuccess) return 0;
    if (threads > fa.maxThreadsPerBlock) return -fa.maxThreadsPerBlock / 32 * 32;
    const int smem = (threads / 32) * kSmemWords * 4;
    cudaFuncSetAttribute(MBE_SEARCH_KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, 32 * kSmemWords * 4);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, MBE_SEARCH_KERNEL, threads, smem) != cudaSuccess) return 0;
    return blocks_per_sm_req < per_sm ? blocks_per_sm_req : per_sm;
}

cudaError_t MBE_VARIANT_LAUNCH(const SearchArgs &a, int blocks, int threads, cudaStream_t stream)
{
    static int smem_set[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    const int smem = (threads / 32) * kSmemWords * 4;
    if (dev >= 0 && dev < 64 && smem_set[dev] < 32 * kSmemWords * 4) {
        cudaError_t e =
            cudaFuncSetAttribute(MBE_SEARCH_KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, 32 * kSmemWords * 4);
        if (e != cudaSuccess) return e;
        smem_set[dev] = 32 * kSmemWords * 4;
    }
    MBE_SEARCH_KERNEL<<<blocks, threads, smem, stream>>>(a);
    return cudaGetLastError();
}

#else

int search_smem_per_warp() { return kSmemWords * 4; }

int search_trace_compiled() { return MBE_TRACE; }

int search_fit_shape(int threads, int blocks_per_sm_req)
{
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, search_kernel) != cudaSuccess) return 0;
    if (threads > fa.maxThreadsPerBlock) return -fa.maxThreadsPerBlock / 32 * 32;
    int smem = (threads / 32) * search_smem_per_warp();
    // the limit is a property of the kernel shared by every launch: keep it at
    // the largest block's need (never lower it for a smaller block)
    cudaFuncSetAttribute(search_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 32 * search_smem_per_warp());
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, search_kernel, threads, smem) != cudaSuccess) return 0;
    // the list and pruned variants must fit the same shape
    const int per_sm_l = search_lists_fit_shape(threads, per_sm);
    if (per_sm_l <= 0) return per_sm_l;
    if (per_sm_l < per_sm) per_sm = per_sm_l;
    const int per_sm_p = search_prune_fit_shape(threads, per_sm);
    if (per_sm_p <= 0) return per_sm_p;
    if (per_sm_p < per_sm) per_sm = per_sm_p;
    return blocks_per_sm_req < per_sm ? blocks_per_sm_req : per_sm;
}

cudaError_t launch_search(const SearchArgs &a, int blocks, int threads, cudaStream_t stream)
{
    if (a.prune) return launch_search_prune(a, blocks, threads, stream);
    if (a.lists) return launch_search_lists(a, blocks, threads, stream);
    // the dynamic shared memory limit is raised once to the largest block
    // (no attribute calls between captured launches)
    static int smem_set[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    const int smem = (threads / 32) * search_smem_per_warp();
    if (dev >= 0 && dev < 64 && smem_set[dev] < 32 * search_smem_per_warp()) {
        cudaError_t e = cudaFuncSetAttribute(search_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             32 * search_smem_per_warp());
        if (e != cudaSuccess) return e;
        smem_set[dev] = 32 * search_smem_per_warp();
    }
    search_kernel<<<blocks, threads, smem, stream>>>(a);
    return cudaGetLastError();
}

#endif

} // namespace mbe
