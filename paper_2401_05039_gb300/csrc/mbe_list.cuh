// Sorted-list search nodes for wide level sets (Section III-D: reverse
// scanning with a lookup table), shared by both search kernels.
//
// A level set L wider than the bitset limit (64 * max_words vertices) is not
// packed into bitset rows. Its frame keeps L, Q and P as plain id lists
// (L ascending, P in pop order) and a node works on the graph's adjacency
// lists directly:
//  - L' = L n N(x) by binary searches of the shorter sorted list in the longer;
//  - every candidate of the node (Q, and P after x) gets its index in the
//    worker's lookup array (`mark`, one entry per U vertex), and the counts
//    c(y) = |N(y) n L'| come from one pass over the lists N(w), w in L'
//    (the reverse scan: iterate over L', not over the candidates);
//  - the maximality check, the maximal expansion and P' / Q' follow from
//    the counts as in Algorithm 1.
// A child whose L' fits the bitset limit is built as a bitset frame of the
// kernel's own layout (from the same reverse scan, setting bits instead of
// counting); a wider child is a list frame again. A root wider than the
// limit starts as a list frame.
//
// This file is included inside each kernel's anonymous namespace after the
// kernel's own definitions (GView, gview, warp_sort_impl, the emit helpers)
// and a declaration of the kernel's bits_from_lists. Its entry points are
// kept out of line and take their worker state by value: they run rarely,
// and inlined they would cost the bitset path registers.
#pragma once

// Header of a list frame: the fields a kernel's generic frame code reads
// (cursor, end, size, parent) sit at the same offsets as in both kernels'
// bitset frame headers; W = 0 marks a list frame.
struct __align__(16) ListHdr {
    int32_t m;      // |L|
    int32_t W;      // 0: list frame
    int32_t nQ;     // |Q| inherited
    int32_t nP;     // candidates to pop, in (count, id) order
    int32_t i;      // next P position to pop
    int32_t end;    // one past the last P position this worker pops
    int32_t root;   // top-level candidate of this subtree
    int32_t graph;  // graph of the subtree
    uint64_t Rsum;  // sum of key_u over R
    int32_t nR;     // |R| stored in the frame (emit mode), else 0
    int32_t depth;  // depth below the root (progress records)
    int64_t bytes;  // size of the frame
    int64_t parent; // offset of the parent frame from the arena base, -1 at the bottom
    int32_t rn;     // |R| (exact when bicliques are written or a minimum |R| is set)
    int32_t pad32_;
    int64_t pad_;
};
static_assert(sizeof(ListHdr) == 80, "list frame header size");

struct ListFrame {
    ListHdr *h;
    int32_t *Lid; // [m] ascending V ids
    int32_t *Qid; // [nQ]
    int32_t *Pid; // [nP] in pop order
    int32_t *R;   // [nR] ascending
};

__device__ __forceinline__ int64_t list_frame_bytes(int m, int nQ, int nP, int nR)
{
    return (int64_t)sizeof(ListHdr) + pad16(4LL * m) + pad16(4LL * nQ) + pad16(4LL * nP) + pad16(4LL * nR);
}

__device__ __forceinline__ ListFrame list_frame_at(char *p, int m, int nQ, int nP)
{
    ListFrame f;
    f.h = reinterpret_cast<ListHdr *>(p);
    char *q = p + sizeof(ListHdr);
    f.Lid = reinterpret_cast<int32_t *>(q);
    q += pad16(4LL * m);
    f.Qid = reinterpret_cast<int32_t *>(q);
    q += pad16(4LL * nQ);
    f.Pid = reinterpret_cast<int32_t *>(q);
    q += pad16(4LL * nP);
    f.R = reinterpret_cast<int32_t *>(q);
    return f;
}

__device__ __forceinline__ ListFrame list_frame_of(char *p)
{
    const ListHdr *h = reinterpret_cast<const ListHdr *>(p);
    return list_frame_at(p, h->m, h->nQ, h->nP);
}

__device__ __forceinline__ bool is_list_frame(const char *p)
{
    return reinterpret_cast<const ListHdr *>(p)->W == 0;
}

// What the list path needs from its worker, passed by value (a reference to
// the worker's whole context would force that context out of registers).
struct ListEnv {
    int lane;
    int32_t *mark;   // lookup array, -1 everywhere between uses
    uint32_t *hist;  // shared [256]: radix-sort histogram
    char *arena;     // the worker's stack base
    char *limit;     // frames must end at or below this address
    int32_t *qsrc, *psrc, *psrc2, *rtmp, *ugid, *lbuf; // scratch lists
    uint64_t *pkey, *pkey2, *urows;
    int64_t ncap, urow_words;
};

// What a list node or root adds to the worker's task totals.
struct ListOut {
    char *child;    // pushed frame, or NULL
    uint64_t cnt, hash, bytes;
    bool abort;
};

// Defined by the including kernel: the bitset child of a list node, a frame
// of the kernel's own layout over L' (ascending ids Lp[0..mp), mp at most
// the bitset limit) with check set Q' (ids Qg[0..nQd)) then P' (sorted keys
// Pk[0..pn)), R' = merge of Ra (na) and Rb (nb), |R'| = rn. Returns the
// frame or NULL (error set).
__device__ __noinline__ char *bits_from_lists(const SearchArgs &a, const ListEnv &e, char *cp, const GView &G,
                                              int graph, int root, int rn, int64_t parent, const int32_t *Lp,
                                              int mp, const int32_t *Qg, int nQd, const uint64_t *Pk, int pn,
                                              uint64_t Rs, const int32_t *Ra, int na, const int32_t *Rb, int nb);

// Bit limit of a bitset level set.
__device__ __forceinline__ int bitset_limit(const SearchArgs &a) { return 64 * a.max_words; }

// out[0..) = A n B for ascending A (na) and B (nb), ascending: every element
// of the shorter list is looked up in the longer one by binary search; hits
// are compacted in order with a warp ballot. Returns |A n B|.
__device__ int list_intersect(int lane, const int32_t *A, int na, const int32_t *B, int nb, int32_t *out)
{
    if (na > nb) {
        const int32_t *t = A;
        A = B;
        B = t;
        const int tn = na;
        na = nb;
        nb = tn;
    }
    int n = 0;
    for (int k0 = 0; k0 < na; k0 += 32) {
        const int k = k0 + lane;
        bool hit = false;
        int32_t x = 0;
        if (k < na) {
            x = A[k];
            int lo = 0, hi = nb;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (B[mid] < x) lo = mid + 1;
                else hi = mid;
            }
            hit = lo < nb && B[lo] == x;
        }
        const unsigned bal = __ballot_sync(kFull, hit);
        if (hit) out[n + __popc(bal & lanemask_lt())] = x;
        n += __popc(bal);
    }
    __syncwarp();
    return n;
}

// Reverse scan over the lists N(w), w = Lw[j] for j < n (V -> U adjacency):
// for every (j, u) with look[u] >= 0, calls f(look[u], j). The pairs are
// flattened across up to 32 consecutive w so that lanes stay busy when the
// lists are short. Returns the number of pairs visited.
template <class F>
__device__ uint64_t reverse_scan(int lane, const GView &G, const int32_t *Lw, int n, const int32_t *look, F f)
{
    uint64_t pairs = 0;
    for (int j0 = 0; j0 < n; j0 += 32) {
        const int j = j0 + lane;
        const bool vj = j < n;
        const int w = vj ? Lw[j] : 0;
        const int wo = vj ? G.v_off[w] : 0;
        const int wd = vj ? G.v_off[w + 1] - wo : 0;
        int incl = wd;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        const int excl = incl - wd;
        pairs += (uint64_t)total;
        for (int p0 = 0; p0 < total; p0 += 32) {
            const int p = p0 + lane;
            const bool vp = p < total;
            int s = 0; // last lane whose segment starts at or before p
#pragma unroll
            for (int b = 16; b > 0; b >>= 1) {
                const int cand = s + b;
                const int ex = __shfl_sync(kFull, excl, cand & 31);
                if (cand < 32 && ex <= p) s = cand;
            }
            const int ws = __shfl_sync(kFull, wo, s);
            const int es = __shfl_sync(kFull, excl, s);
            if (vp) {
                const int u = G.v_adj[ws + (p - es)];
                const int k = look[u];
                if (k >= 0) f(k, j0 + s);
            }
        }
    }
    __syncwarp();
    return pairs;
}

// Pushes a list frame at cp holding L = Lw[0..m), Q = Qg[0..nQ), P = the
// ids in the low bits of the sorted keys Pk[0..nP), R = the merge of Ra (na)
// and Rb (nb) (emit mode). The caller checked the stack limit.
__device__ void write_list_frame(const SearchArgs &a, const ListEnv &e, char *cp, const int32_t *Lw, int m, const int32_t *Qg,
                                 int nQ, const uint64_t *Pk, int nP, const int32_t *Ra, int na, const int32_t *Rb,
                                 int nb, uint64_t Rsum, int root, int graph, int i0, int i1, int depth,
                                 int64_t parent, int64_t bytes, int rn)
{
    const int lane = e.lane;
    ListFrame D = list_frame_at(cp, m, nQ, nP);
    const uint64_t id_mask = (1ULL << a.key_shift) - 1;
    for (int k = lane; k < m; k += 32) D.Lid[k] = Lw[k];
    for (int k = lane; k < nQ; k += 32) D.Qid[k] = Qg[k];
    for (int k = lane; k < nP; k += 32) D.Pid[k] = (int32_t)(Pk[k] & id_mask);
    const int nR = a.emit ? na + nb : 0;
    if (a.emit) emit::merge_into(lane, Ra, na, Rb, nb, D.R);
    if (lane == 0) {
        ListHdr h;
        h.m = m;
        h.W = 0;
        h.nQ = nQ;
        h.nP = nP;
        h.i = i0;
        h.end = i1;
        h.root = root;
        h.graph = graph;
        h.Rsum = Rsum;
        h.nR = nR;
        h.depth = depth;
        h.bytes = bytes;
        h.parent = parent;
        h.rn = rn;
        h.pad32_ = 0;
        h.pad_ = 0;
        *D.h = h;
    }
    __syncwarp();
}

// The top-level iteration for a root r whose degree d exceeds the bitset
// limit: L' = N(r) (ascending), the candidates N2(r) \ {r} with their counts
// |N(u) n N(r)| from one reverse scan, the check against the earlier-ranked
// candidates, the expansion by the later-ranked ones, emit, and the level-1
// list frame at the bottom of the stack (out.child). The caller counts the
// node itself.
__device__ __noinline__ ListOut list_root(const SearchArgs &a, const ListEnv e, const GView G, int r, int graph,
                                          int part, int parts)
{
    ListOut out{nullptr, 0, 0, 0, false};
    const int lane = e.lane;
    const int ro = G.u_off[r];
    const int d = G.u_off[r + 1] - ro;
    const bool first = part == 0;
    const int32_t *Ln = G.u_adj + ro;
    int32_t *mark = e.mark;
    int32_t *cnt = e.psrc2;

    // Discovery: local ids for N2(r) \ {r} (ugid) by the flattened pass of
    // the bitset path, counting instead of setting bits.
    int nc = 0;
    uint64_t pairs_total = 0;
    for (int j0 = 0; j0 < d && !out.abort; j0 += 32) {
        const int j = j0 + lane;
        const bool vj = j < d;
        const int w = vj ? Ln[j] : 0;
        const int wo = vj ? G.v_off[w] : 0;
        const int wd = vj ? G.v_off[w + 1] - wo : 0;
        int incl = wd;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        const int excl = incl - wd;
        pairs_total += (uint64_t)total;
        for (int p0 = 0; p0 < total; p0 += 32) {
            const int p = p0 + lane;
            const bool vp = p < total;
            int s = 0;
#pragma unroll
            for (int b = 16; b > 0; b >>= 1) {
                const int cand = s + b;
                const int ex = __shfl_sync(kFull, excl, cand & 31);
                if (cand < 32 && ex <= p) s = cand;
            }
            const int ws = __shfl_sync(kFull, wo, s);
            const int es = __shfl_sync(kFull, excl, s);
            const int u = vp ? G.v_adj[ws + (p - es)] : -1;
            const bool take = vp && u != r;
            const int cur = take ? mark[u] : 0;
            const bool need = take && cur < 0;
            const unsigned grp = __match_any_sync(kFull, need ? u : -2 - lane);
            const int leader_lane = __ffs(grp) - 1;
            const bool leader = need && leader_lane == lane;
            const unsigned lb = __ballot_sync(kFull, leader);
            const int newid = nc + __popc(lb & lanemask_lt());
            const int nnew = __popc(lb);
            if (nc + nnew > e.ncap) {
                if (lane == 0) set_error(a, kErrArena);
                out.abort = true;
                break;
            }
            if (leader) {
                mark[u] = newid;
                e.ugid[newid] = u;
                cnt[newid] = 0;
            }
            nc += nnew;
            __syncwarp();
            const int from = __shfl_sync(kFull, newid, leader_lane);
            const int id = need ? from : cur;
            if (take) atomicAdd(&cnt[id], 1);
        }
    }
    __syncwarp();
    for (int k = lane; k < nc; k += 32) mark[e.ugid[k]] = -1;
    __syncwarp();
    if (first) out.bytes += 4ULL * ((uint64_t)d + pairs_total);
    if (out.abort) return out;

    // Classify: earlier-ranked candidates (degree, id) < (d, r) form Q.
    uint64_t rsum = 0;
    int qn = 0, pn = 0, nfull = 0;
    for (int t0 = 0; t0 < nc; t0 += 32) {
        const int k = t0 + lane;
        const bool valid = k < nc;
        int u = 0, du = 0, ck = 0;
        if (valid) {
            u = e.ugid[k];
            du = G.u_off[u + 1] - G.u_off[u];
            ck = cnt[k];
        }
        // earlier-ranked candidates were popped before r (those below the size
        // filter never are)
        const bool earlier = du < d || (du == d && u < r);
        const bool ql = valid && earlier && du >= a.min_l;
        if (__ballot_sync(kFull, ql && ck == d)) return out; // r's node is not maximal
        const bool full = valid && !earlier && ck == d;
        const bool ppart = valid && !earlier && ck < d && ck >= a.min_l;
        if (full) rsum += key_u(u);
        if (a.emit || a.min_r > 1) {
            const unsigned fb = __ballot_sync(kFull, full);
            if (a.emit && full) e.rtmp[nfull + __popc(fb & lanemask_lt())] = u;
            nfull += __popc(fb);
        }
        const unsigned qb = __ballot_sync(kFull, ql);
        if (ql) e.qsrc[qn + __popc(qb & lanemask_lt())] = u;
        qn += __popc(qb);
        const unsigned pb = __ballot_sync(kFull, ppart);
        if (ppart) {
            const int q = pn + __popc(pb & lanemask_lt());
            e.pkey[q] = ((uint64_t)ck << a.key_shift) | (uint64_t)(uint32_t)u;
            e.psrc[q] = q;
        }
        pn += __popc(pb);
    }
    rsum = warp_sum64(rsum);
    const uint64_t Rs = key_u(r) + rsum;
    const bool pass = 1 + nfull >= a.min_r; // d >= min_l already
    if (first && pass) {
        uint64_t ls = 0;
        for (int j = lane; j < d; j += 32) ls += key_v(Ln[j]);
        ls = warp_sum64(ls);
        out.cnt += 1;
        out.hash += splitmix(Rs + ls);
    }
    if (a.emit) {
        // R' = {r} and the candidates that joined it, ascending; L' = N(r)
        if (lane == 0) e.rtmp[nfull] = r;
        __syncwarp();
        emit::sort_ids(lane, e.hist, e.rtmp, e.psrc2, nfull + 1, a.key_shift);
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
                for (int k = lane; k < nR; k += 32) o[2 + k] = e.rtmp[k];
                for (int k = lane; k < d; k += 32) o[2 + nR + k] = Ln[k];
                __syncwarp();
            }
        }
    }
    if (pn == 0 || d - 1 < a.min_l || 1 + nfull + pn < a.min_r) return out;

    const int nR = a.emit ? 1 + nfull : 0;
    const int64_t sz = list_frame_bytes(d, qn, pn, nR);
    if (e.arena + sz > e.limit) {
        if (lane == 0) set_error(a, kErrArena);
        out.abort = true;
        return out;
    }
    const int key_bits = a.key_shift + (32 - __clz(d));
    warp_sort_impl(lane, e.hist, e.pkey, e.psrc, e.pkey2, e.psrc2, pn, key_bits);
    const int i0 = (int)(((int64_t)pn * part) / parts), i1 = (int)(((int64_t)pn * (part + 1)) / parts);
    write_list_frame(a, e, e.arena, Ln, d, e.qsrc, qn, e.pkey, pn, e.rtmp, nR, nullptr, 0, Rs, r, graph, i0, i1, 1, -1,
                     sz, 1 + nfull);
    out.child = e.arena;
    return out;
}

// One iteration of Algorithm 1's while loop on the list frame at fp (see
// the top of this file). A child whose L' fits the bitset limit is built by
// the including kernel's bits_from_lists, which receives L' (ascending ids),
// Q' (ids), P' (sorted keys), R' and the stack address; a wider child is
// pushed as a list frame here. The caller counts the node itself.
__device__ __noinline__ ListOut list_node(const SearchArgs &a, const ListEnv e, char *fp)
{
    ListOut out{nullptr, 0, 0, 0, false};
    const int lane = e.lane;
    ListFrame F = list_frame_of(fp);
    const int m = F.h->m, nQ = F.h->nQ, nP = F.h->nP, i = F.h->i;
    __syncwarp(); // every lane has read the header before lane 0 advances the cursor
    if (lane == 0) F.h->i = i + 1;
    const GView G = gview(a, F.h->graph);
    const int x = F.Pid[i];
    const int xo = G.u_off[x], dx = G.u_off[x + 1] - xo;

    // Step 2: L' = L n N(x)
    int32_t *Lp = e.lbuf;
    const int mp = list_intersect(lane, F.Lid, m, G.u_adj + xo, dx, Lp);

    // Counts of every candidate by one reverse scan over L': Q (the inherited
    // Q, then the P entries popped before x) at indices [0, nq), P after x at
    // [nq, nq + nrest).
    const int nq = nQ + i, nrest = nP - i - 1, nx = nq + nrest;
    if (nx > e.ncap) {
        if (lane == 0) set_error(a, kErrInternal);
        out.abort = true;
        return out;
    }
    int32_t *mark = e.mark;
    int32_t *cnt = e.psrc2;
    auto cand = [&](int k) { return k < nQ ? F.Qid[k] : F.Pid[k < nq ? k - nQ : k - nq + i + 1]; };
    for (int k = lane; k < nx; k += 32) {
        mark[cand(k)] = k;
        cnt[k] = 0;
    }
    __syncwarp();
    reverse_scan(lane, G, Lp, mp, mark, [&](int k, int) { atomicAdd(&cnt[k], 1); });
    for (int k = lane; k < nx; k += 32) mark[cand(k)] = -1;
    __syncwarp();

    // Step 3: maximality check against Q
    bool rejected = false;
    for (int k0 = 0; k0 < nq && !rejected; k0 += 32) {
        const int k = k0 + lane;
        rejected = __ballot_sync(kFull, k < nq && cnt[k] == mp) != 0;
    }
    {
        // algorithmic bytes, as for a bitset frame of the same sets
        const uint64_t W = (uint64_t)((m + 63) >> 6), q = (uint64_t)nq, rows = W * q,
                       cols = (uint64_t)mp * ((q + 63) >> 6);
        out.bytes += 8ULL * (W + (rows < cols ? rows : cols) + (rejected ? 0ULL : W * (uint64_t)nrest));
    }
    if (rejected) return out;

    // Step 4: maximal expansion over P after x; Q' from the counts of Q
    uint64_t rsum = 0;
    int pn = 0, nfull = 0, qn = 0;
    for (int k0 = 0; k0 < nx; k0 += 32) {
        const int k = k0 + lane;
        const bool valid = k < nx;
        const int ck = valid ? cnt[k] : 0;
        const int u = valid ? cand(k) : 0;
        const bool isq = valid && k < nq;
        const bool qpart = isq && ck > 0;
        const bool full = valid && !isq && ck == mp;
        const bool part = valid && !isq && ck > 0 && ck < mp && ck >= a.min_l;
        if (full) rsum += key_u(u);
        if (a.emit || a.min_r > 1) {
            const unsigned fb = __ballot_sync(kFull, full);
            if (a.emit && full) e.rtmp[nfull + __popc(fb & lanemask_lt())] = u;
            nfull += __popc(fb);
        }
        const unsigned qb = __ballot_sync(kFull, qpart);
        if (qpart) e.qsrc[qn + __popc(qb & lanemask_lt())] = u;
        qn += __popc(qb);
        const unsigned pb = __ballot_sync(kFull, part);
        if (part) {
            const int q = pn + __popc(pb & lanemask_lt());
            e.pkey[q] = ((uint64_t)ck << a.key_shift) | (uint64_t)(uint32_t)u;
            e.psrc[q] = q;
        }
        pn += __popc(pb);
    }
    rsum = warp_sum64(rsum);
    const uint64_t Rs = F.h->Rsum + key_u(x) + rsum;
    uint64_t ls = 0;
    for (int k = lane; k < mp; k += 32) ls += key_v(Lp[k]);
    ls = warp_sum64(ls);
    // size filter (1, 1 by default: every biclique passes)
    const int rn = F.h->rn + 1 + nfull;
    const bool pass = rn >= a.min_r && mp >= a.min_l;
    if (pass) {
        out.cnt += 1;
        out.hash += splitmix(Rs + ls);
    }

    if (a.emit) {
        // B = {x} and the candidates that joined R', ascending
        if (lane == 0) e.rtmp[nfull] = x;
        __syncwarp();
        emit::sort_ids(lane, e.hist, e.rtmp, e.psrc2, nfull + 1, a.key_shift);
        const int nR = F.h->nR + nfull + 1;
        int64_t rec = 0;
        const int64_t pos = pass ? emit::reserve(a, lane, 2 + (int64_t)nR + mp, &rec) : -1;
        if (pos >= 0) {
            int32_t *o = a.out_ids + pos;
            if (lane == 0) {
                a.out_offsets[rec] = pos;
                o[0] = nR;
                o[1] = mp;
            }
            emit::merge_into(lane, F.R, F.h->nR, e.rtmp, nfull + 1, o + 2);
            for (int k = lane; k < mp; k += 32) o[2 + nR + k] = Lp[k];
            __syncwarp();
        }
    }
    // the child's level sets are smaller than L' and its R within R' u P'
    if (pn == 0 || mp - 1 < a.min_l || rn + pn < a.min_r) return out;

    // Child: P' in pop order (count, id)
    const int key_bits = a.key_shift + (32 - __clz(mp));
    warp_sort_impl(lane, e.hist, e.pkey, e.psrc, e.pkey2, e.psrc2, pn, key_bits);
    char *cp = fp + F.h->bytes;
    const int nb = a.emit ? nfull + 1 : 0;
    if (mp <= bitset_limit(a)) {
        out.child = bits_from_lists(a, e, cp, G, F.h->graph, F.h->root, rn, fp - e.arena, Lp, mp, e.qsrc, qn, e.pkey,
                                    pn, Rs, F.R, F.h->nR, e.rtmp, nb);
        out.abort = out.child == nullptr;
        return out;
    }
    const int nR = a.emit ? F.h->nR + nb : 0;
    const int64_t sz = list_frame_bytes(mp, qn, pn, nR);
    if (cp + sz > e.limit) {
        if (lane == 0) set_error(a, kErrArena);
        out.abort = true;
        return out;
    }
    write_list_frame(a, e, cp, Lp, mp, e.qsrc, qn, e.pkey, pn, F.R, F.h->nR, e.rtmp, nb, Rs, F.h->root, F.h->graph, 0,
                     pn, F.h->depth + 1, fp - e.arena, sz, rn);
    out.child = cp;
    return out;
}
