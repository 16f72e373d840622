// fsm_extend.cuh -- the two-vertex extension kernel (one level l -> l+2).
//
// Work: every (frontier embedding s, key position i) "unit" owns the pieces keyed at v = s[i]:
//   centre pieces  {v, a, b}, a < b both in N(v): the wedge a-v-b, and the triangle if a ~ b;
//   end pieces     {v, a, b}, a in N(v), b in N(a) \ {v}: the wedge v-a-b centred at a.
// Together these are every connected size-3 subgraph containing v (edge-induced); in
// vertex-induced mode a closed triple yields only its triangle.  Joining s with a piece t on v
// is Section 4.1's two-vertex exploration, equivalent to the hash join of Section 4.2 on the
// column holding v; the piece list is generated from the CSR instead of being stored.
//
// Per join: require s and t to share only v (Algorithm 1's first test); read the cross
// adjacencies between s \ {v} and t \ {v}; for each subset of them (edge-induced) or all of them
// (vertex-induced) prune when a joining-point triple {v, s[p], t[q]} is connected with an
// infrequent size-3 pattern (Section 4.5), keep the join only when smallest-vertex-first
// dissection returns exactly (t, s) (Algorithm 1), and form its index-based quick pattern key
// (Section 4.4).  The pass template parameter says what an accepted join does:
//   PASS_COUNT   insert the key into the quick-pattern table and count it;
//   PASS_DOMAIN  set the MNI domain bits of its pattern's orbits (Definition 2);
//   PASS_EMIT    write it, permuted into canonical order, to the next frontier;
//   PASS_FUSED   (last level, k <= 7) count it and set the MNI domain bits of its pattern's
//                orbits in the same enumeration: the lane that first meets a quick pattern
//                canonicalises it, claims its pattern's orbit bitmaps (one CAS on the pattern's
//                entry in a table of canonical codes) and publishes the bitmap word offset of
//                every local position; nothing waits on another lane.
//
// Scheduling: the pieces of a batch of units form one index space [0, total) (exclusive prefix
// `unit_base`); warps take fixed-size chunks of it from an atomic counter, so hub vertices
// with millions of pieces are split across many warps and light units share a warp.
#pragma once
#include "fsm_canon7.cuh"

namespace fsm {

enum { PASS_COUNT = 0, PASS_DOMAIN = 1, PASS_EMIT = 2, PASS_FUSED = 3 };

struct QPTab {
    unsigned long long *keys;      // [cap], FSM_EMPTY_KEY when free
    unsigned long long *count;     // [cap] accepted joins per key
    int32_t *pattern;              // [cap] pattern id of the key (after canonicalisation)
    uint64_t *perm;                // [cap] local vertex h -> canonical position, 4 bits each (nib_get)
    uint64_t mask;                 // cap - 1 (cap a power of two)
    unsigned long long *used;      // occupied slots
    unsigned long long max_used;   // overflow threshold (load factor 1/2)
};

struct ExtArgs {
    DevGraph g;
    int mode;                      // 0 edge-induced, 1 vertex-induced
    // frontier batch: embeddings [e0, e0 + ne) of an SoA array with stride fN
    const int32_t *fv;
    const int32_t *fpid;
    int64_t fN, e0, ne;
    const int64_t *unit_base;      // [ne*L + 1] exclusive prefix of pieces per unit
    int64_t total;                 // pieces in this batch; < 0: read unit_base[ne*L] on the device
    int64_t nchunks;               // ignored when total < 0
    int32_t chunk;                 // pieces per chunk; <= 0 with total < 0: sized on the device
    unsigned long long *chunk_ctr;
    // size-l pattern table (frequent patterns of the level being extended)
    const uint64_t *pat_adj;       // [P] 8 adjacency rows (one byte each) over canonical positions
    // frequent size-3 patterns, by piece index; NULL at level 1 (nothing is known yet)
    const uint8_t *piece_freq;
    // optional restriction of the pieces joined (exact recount of sampled mining); NULL = all
    const uint8_t *piece_sel;
    QPTab qp;
    // domains (PASS_DOMAIN)
    const uint8_t *live;           // [P'] pattern has domains
    const uint64_t *orbit;         // [P'] orbit word: representative per canonical position
    const int64_t *dom_off;        // [P'*FSM_MAXK] word offset per orbit representative
    uint32_t *dom;
    const int64_t *slot_base;      // [cap*FSM_MAXK] bitmap word offset per (key slot, local position), -1 none
    // emission (PASS_EMIT)
    const int32_t *newid;          // [P'] id among frequent patterns, -1 otherwise
    int32_t *out_v;                // SoA [K][out_N]
    int32_t *out_pid;
    int64_t out_N;
    unsigned long long *out_cursor;
    unsigned long long *stats;     // [0] joins tested, [1] joins accepted, [2] pieces enumerated
    // one-pass last level (PASS_FUSED): a table of canonical codes (packed by pack_code) with the
    // pool word offset + 1 of each pattern's orbit bitmaps (0 = not yet claimed), and the bitmap
    // word offset of every (key slot, local position), -1 until published
    const uint64_t *pat_lab;       // [P] 8 label bytes of the size-l patterns
    unsigned long long *code_keys; // [code_mask + 1], FSM_EMPTY_KEY when free
    unsigned long long *code_off;  // [code_mask + 1]
    uint64_t code_mask;
    long long *slot_off;           // [cap * 8]
    uint32_t *pool;
    unsigned long long *pool_top;
    unsigned long long pool_words;
    const int32_t *cls_size;
    int explore;                   // exploration variant (quick-pattern key layout)
    int level;                     // L, the size of the embeddings extended
    // sampled last level (pieces come from the kept edges in g.prow / g.pcol)
    int sampled;
    // sampling quotas (variant FSM_EXPLORE_TV_QUOTA): candidate pieces per unit (0 = all) and,
    // when an edge list is joined, edges per key vertex (0 = all); draws seeded by qseed
    int64_t quota;
    int64_t edge_quota;
    uint64_t qseed;
    int debug;                     // option "debug": bounds-check decoded indices, flag and skip
    uint64_t time_limit_ns;        // option "time_limit_ms" in ns (0 = none), from *time_start
    const unsigned long long *time_start;   // the call's start on the device's global timer
    int *err;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int64_t last_le(const int64_t *base, int64_t lo, int64_t hi, int64_t x) {
    // largest u in [lo, hi] with base[u] <= x (base[lo] <= x assumed)
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (base[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Linear probing stops after FSM_MAX_PROBES slots: at load <= 1/2 a run that long means the
// table is too small, so the pass is flagged, abandoned and repeated with a larger table.
#define FSM_MAX_PROBES 256

__device__ __forceinline__ int64_t qp_insert(const QPTab &t, uint64_t key, int *err) {
    uint64_t h = mix64(key) & t.mask;
    for (uint64_t probe = 0; probe <= t.mask && probe < FSM_MAX_PROBES; ++probe) {
        unsigned long long cur = __ldcg(t.keys + h);
        if (cur == key) return (int64_t)h;
        if (cur == FSM_EMPTY_KEY) {
            unsigned long long old = atomicCAS(t.keys + h, FSM_EMPTY_KEY, key);
            if (old == FSM_EMPTY_KEY) {
                unsigned long long u = atomicAdd(t.used, 1ull);
                if (u >= t.max_used) atomicOr(err, FSM_ERR_QP_OVERFLOW);
                return (int64_t)h;
            }
            if (old == key) return (int64_t)h;
        }
        h = (h + 1) & t.mask;
    }
    atomicOr(err, FSM_ERR_QP_OVERFLOW);
    return -1;
}

__device__ __forceinline__ int64_t qp_find(const QPTab &t, uint64_t key) {
    uint64_t h = mix64(key) & t.mask;
    for (uint64_t probe = 0; probe <= t.mask; ++probe) {
        unsigned long long cur = __ldg(t.keys + h);
        if (cur == key) return (int64_t)h;
        if (cur == FSM_EMPTY_KEY) return -1;
        h = (h + 1) & t.mask;
    }
    return -1;
}

// Is u ~ w, given both row ranges: binary search in the shorter list.
__device__ __forceinline__ bool adj_rows(const int32_t *col, int32_t bu, int32_t eu, int32_t u, int32_t bw,
                                         int32_t ew, int32_t w) {
    int32_t lo, end, x;
    if (eu - bu <= ew - bw) { lo = bu; end = eu; x = w; } else { lo = bw; end = ew; x = u; }
    int32_t hi = end;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (__ldg(col + mid) < x) lo = mid + 1; else hi = mid;
    }
    return lo < end && __ldg(col + lo) == x;
}

template <int L>
__device__ __forceinline__ bool in_s(const int32_t (&S)[L], int32_t x) {
    bool r = false;
#pragma unroll
    for (int p = 0; p < L; ++p) r |= (S[p] == x);
    return r;
}

struct Tally { unsigned long long tested, accepted; };

// Local vertex of smallest id among the bits of m (four vertices).
FSM_HD int argmin4(uint32_t m, const int32_t (&gid)[4]) {
    int b = -1;
#pragma unroll
    for (int h = 0; h < 4; ++h)
        if ((m >> h & 1u) && (b < 0 || gid[h] < gid[b])) b = h;
    return b;
}

// Algorithm 1 for a four-vertex join (s = local 0, 1 with key position i; piece vertices 2, 3),
// as a closed form.  The greedy round from the smallest vertex m always succeeds for four
// vertices (the one vertex left is adjacent to the connected 3-set), so the dissection is that
// round: the 3-set {m, n1, n2}, n1 the smallest neighbour of m and n2 the smallest further
// neighbour of {m, n1}, joined at its smallest vertex adjacent to the fourth.  The join is kept
// when that 3-set is the piece and the join vertex is s[i] -- what dissect3 returns, without
// its loops.
FSM_HD bool dissect4_keeps(const int32_t (&gid)[4], const uint32_t (&adj)[4], int i) {
    const int m = argmin4(15u, gid);
    const int n1 = argmin4(adj[m], gid);
    const int n2 = argmin4((adj[m] | adj[n1]) & ~((1u << m) | (1u << n1)), gid);
    const uint32_t l = (1u << m) | (1u << n1) | (1u << n2);
    if (l != ((1u << i) | 12u)) return false;
    return argmin4(adj[1 - i] & l, gid) == i;
}

// neighbour-adjacency masks of single-unit chunks: key vertices of degree up to 32 * this
#define FSM_MASK_WORDS 64
// masks of multi-unit chunks: at most this many units (two words per other position each)
#define FSM_MASK_UNITS (FSM_MASK_WORDS / 2)

// Per-warp aggregation of quick-pattern counts (PASS_COUNT).  Within one chunk the same few
// keys repeat (one unit, one pattern, a few piece labels), so each warp sums them in its own
// shared-memory table and flushes the table to the global one at the end of the chunk; keys
// that find no free slot go straight to the global table.  Hot keys (the dominant label
// patterns) would otherwise serialise on one global counter.
#define FSM_WARP_SLOTS 128
#define FSM_SMEM_PROBES 16
struct CountCache {
    unsigned long long key[8][FSM_WARP_SLOTS];
    unsigned long long cnt[8][FSM_WARP_SLOTS];
    long long slot[8][FSM_WARP_SLOTS];   // global slot of the key, -1 until resolved (PASS_FUSED)
};
// PASS_COUNT launches allocate only key and cnt: more of the SM's shared storage stays L1.
#define FSM_COUNT_SMEM (2 * 8 * FSM_WARP_SLOTS * sizeof(unsigned long long))

// Count n more joins of key through the warp's table; returns the key's global slot (resolved
// once per table entry; a race resolves it twice to the same value).
__device__ __forceinline__ int64_t count_key_slot(const ExtArgs &A, CountCache *cc, uint64_t key, unsigned n) {
    const int w = threadIdx.x >> 5;
    uint32_t h = (uint32_t)mix64(key) & (FSM_WARP_SLOTS - 1);
    for (int probe = 0; probe < FSM_SMEM_PROBES; ++probe) {
        unsigned long long cur = cc->key[w][h];
        if (cur == FSM_EMPTY_KEY) cur = atomicCAS(&cc->key[w][h], FSM_EMPTY_KEY, key);
        if (cur == FSM_EMPTY_KEY || cur == key) {
            atomicAdd(&cc->cnt[w][h], (unsigned long long)n);
            long long s = ((volatile long long *)cc->slot[w])[h];
            if (s < 0) {
                s = qp_insert(A.qp, key, A.err);
                ((volatile long long *)cc->slot[w])[h] = s;
            }
            return s;
        }
        h = (h + 1) & (FSM_WARP_SLOTS - 1);
    }
    int64_t slot = qp_insert(A.qp, key, A.err);
    if (slot >= 0) atomicAdd(A.qp.count + slot, (unsigned long long)n);
    return slot;
}

__device__ __forceinline__ void count_key(const ExtArgs &A, CountCache *cc, uint64_t key, unsigned n) {
    const int w = threadIdx.x >> 5;
    uint32_t h = (uint32_t)mix64(key) & (FSM_WARP_SLOTS - 1);
    for (int probe = 0; probe < FSM_SMEM_PROBES; ++probe) {
        unsigned long long cur = cc->key[w][h];
        if (cur == FSM_EMPTY_KEY) cur = atomicCAS(&cc->key[w][h], FSM_EMPTY_KEY, key);
        if (cur == FSM_EMPTY_KEY || cur == key) {
            atomicAdd(&cc->cnt[w][h], (unsigned long long)n);
            return;
        }
        h = (h + 1) & (FSM_WARP_SLOTS - 1);
    }
    int64_t slot = qp_insert(A.qp, key, A.err);
    if (slot >= 0) atomicAdd(A.qp.count + slot, (unsigned long long)n);
}

// warp-synchronous: every lane of the warp calls it
template <bool SLOTS>
__device__ __forceinline__ void flush_warp_counts(const ExtArgs &A, CountCache *cc) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncwarp();
    for (int x = lane; x < FSM_WARP_SLOTS; x += 32) {
        const unsigned long long key = cc->key[w][x];
        if (key == FSM_EMPTY_KEY) continue;
        int64_t slot = SLOTS ? cc->slot[w][x] : -1;
        if (slot < 0) slot = qp_insert(A.qp, key, A.err);
        if (slot >= 0) atomicAdd(A.qp.count + slot, cc->cnt[w][x]);
        cc->key[w][x] = FSM_EMPTY_KEY;
        cc->cnt[w][x] = 0ull;
        if (SLOTS) cc->slot[w][x] = -1;
    }
    __syncwarp();
}

// ---- one-pass last level: publication of per-slot bitmap offsets (gpu-scope release/acquire)
__device__ __forceinline__ long long ld_acquire_s64(const long long *p) {
    long long v;
    asm volatile("ld.acquire.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ long long ld_relaxed_s64(const long long *p) {
    long long v;
    asm volatile("ld.relaxed.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_s64(long long *p, long long v) {
    asm volatile("st.release.gpu.global.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_s64(long long *p, long long v) {
    asm volatile("st.relaxed.gpu.global.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// First sight of a quick pattern in the one-pass last level: canonicalise the graph its key
// denotes, find or claim its pattern's entry in the code table, claim the pattern's orbit
// bitmaps from the pool unless another lane already did (one CAS decides; a loser's pool words
// stay unused), and publish the bitmap word offset of each local position -- position 0 last,
// with release semantics, so a reader that sees it set sees the others.  Lanes racing on one key
// compute and write the same values.  On a full table or pool the error word says so and nothing
// is published; the host then runs the last level as two passes.
struct ResolveArgs {
    const uint64_t *pat_lab, *pat_adj;
    const int32_t *cls_size;
    unsigned long long *code_keys, *code_off, *pool_top;
    uint64_t code_mask;
    unsigned long long pool_words;
    long long *slot_off;
    int *err;
    int explore, level;
};

static __device__ __noinline__ void resolve_slot(const ResolveArgs A, int64_t slot, uint64_t key) {
    // K <= 7 here: the compact words of fsm_canon7.cuh
    int K, lab[8], rep[8];
    uint32_t adj[8];
    key_graph7(A.explore, A.level, key, A.pat_lab, A.pat_adj, K, lab, adj);
    unsigned long long clab;
    uint32_t cadj, inv;
    canonicalise7(K, lab, adj, clab, cadj, inv);
    orbit_reps7(K, clab, cadj, rep);
    int64_t pre[8], words = 0;
    for (int c = 0; c < K; ++c) {
        pre[c] = words;
        if (rep[c] == c) words += ((int64_t)__ldg(A.cls_size + ((clab >> (8 * (7 - c))) & 0xff)) + 31) / 32;
    }
    const uint64_t pk = pack_code7(K, clab, cadj);
    uint64_t h = mix64(pk) & A.code_mask;
    int64_t ci = -1;
    for (int probe = 0; probe < FSM_MAX_PROBES; ++probe) {
        unsigned long long cur = __ldcg(A.code_keys + h);
        if (cur == FSM_EMPTY_KEY) cur = atomicCAS(A.code_keys + h, FSM_EMPTY_KEY, pk);
        if (cur == FSM_EMPTY_KEY || cur == pk) { ci = (int64_t)h; break; }
        h = (h + 1) & A.code_mask;
    }
    if (ci < 0) { atomicOr(A.err, FSM_ERR_CODE_FULL); return; }
    unsigned long long off = __ldcg(A.code_off + ci);
    if (off == 0ull) {
        const unsigned long long res = atomicAdd(A.pool_top, (unsigned long long)words);
        if (res + (unsigned long long)words > A.pool_words) { atomicOr(A.err, FSM_ERR_POOL); return; }
        const unsigned long long old = atomicCAS(A.code_off + ci, 0ull, res + 1ull);
        off = old ? old : res + 1ull;
    }
    long long *so = A.slot_off + slot * 8;
    for (int hh = K - 1; hh >= 0; --hh) {
        const long long v = (long long)(off - 1ull) + pre[rep[(inv >> (3 * hh)) & 7]];
        if (hh) st_relaxed_s64(so + hh, v); else st_release_s64(so, v);
    }
}

// One accepted join: act according to PASS.
// Per-lane memory of bitmap words already set (PASS_DOMAIN, PASS_FUSED): the last word of a piece
// vertex with its bits, and per position of s the last bitmap offset set for it (valid within
// one unit: s and so its vertices' ranks are fixed there; -1 after a unit change).
struct DomCache {
    uint32_t *w;
    uint32_t bits;
    int64_t soff[FSM_MAXL];
};

template <int L, int K, int PASS>
__device__ __forceinline__ void accept(const ExtArgs &A, CountCache *cc, DomCache &dc, uint64_t key,
                                       const int32_t (&gid)[K], const int32_t (&rk)[L]) {
    if (PASS == PASS_COUNT) {
        const unsigned act = __activemask();
        const unsigned grp = __match_any_sync(act, key);
        const int lane = threadIdx.x & 31;
        if (lane == __ffs(grp) - 1) count_key(A, cc, key, __popc(grp));
        return;
    }
    if (PASS == PASS_FUSED) {
        // count the key (warp-aggregated), then set its orbits' bits as the domain pass does
        const unsigned act = __activemask();
        const unsigned grp = __match_any_sync(act, key);
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(grp) - 1;
        // the leader counts the key, resolves it on first sight, and reads its offsets once; the
        // lanes of the group receive them by shuffle
        long long off[K];
#pragma unroll
        for (int h = 0; h < K; ++h) off[h] = -1;
        if (lane == leader) {
            const long long slot = count_key_slot(A, cc, key, __popc(grp));
            if (slot >= 0) {
                const long long *so = A.slot_off + slot * 8;
                long long o0 = ld_acquire_s64(so);
                if (o0 < 0) {
                    const ResolveArgs R{A.pat_lab, A.pat_adj, A.cls_size, A.code_keys, A.code_off, A.pool_top,
                                        A.code_mask, A.pool_words, A.slot_off, A.err, A.explore, A.level};
                    resolve_slot(R, slot, key);
                    o0 = ld_acquire_s64(so);
                }
                if (o0 >= 0) {
                    off[0] = o0;
#pragma unroll
                    for (int h = 1; h < K; ++h) off[h] = ld_relaxed_s64(so + h);
                }
            }
        }
#pragma unroll
        for (int h = 0; h < K; ++h) off[h] = __shfl_sync(grp, off[h], leader);
        // table overflow (the pass is repeated with a larger table), or pool or code table full
        // (the level is redone in two passes): nothing to set
        if (off[0] < 0) return;
#pragma unroll
        for (int h = 0; h < L; ++h) {
            if (off[h] == dc.soff[h]) continue;
            dc.soff[h] = off[h];
            uint32_t *w = A.pool + off[h] + (rk[h] >> 5);
            const uint32_t bit = 1u << (rk[h] & 31);
            if (!(__ldcg(w) & bit)) atomicOr(w, bit);
        }
#pragma unroll
        for (int h = L; h < K; ++h) {
            const int32_t r = __ldg(A.g.rank + gid[h]);
            uint32_t *w = A.pool + off[h] + (r >> 5);
            const uint32_t bit = 1u << (r & 31);
            if (w == dc.w && (dc.bits & bit)) continue;
            atomicOr(w, bit);
            if (w != dc.w) { dc.w = w; dc.bits = 0; }
            dc.bits |= bit;
        }
        return;
    }
    int64_t slot = qp_find(A.qp, key);
    if (slot < 0) { atomicOr(A.err, FSM_ERR_QP_MISSING); return; }
    if (PASS == PASS_DOMAIN) {
        // one load per position: the bitmap of the orbit this key's position h lands in
        const int64_t *sb = A.slot_base + slot * FSM_MAXK;
        if (__ldg(sb) < 0) return;   // pattern without domains
#pragma unroll
        for (int h = 0; h < L; ++h) {
            // a vertex of s: the same word for every join of this unit into the same orbit
            const int64_t off = __ldg(sb + h);
            if (off == dc.soff[h]) continue;
            dc.soff[h] = off;
            uint32_t *w = A.dom + off + (rk[h] >> 5);
            const uint32_t bit = 1u << (rk[h] & 31);
            if (!(__ldcg(w) & bit)) atomicOr(w, bit);
        }
#pragma unroll
        for (int h = L; h < K; ++h) {
            const int64_t off = __ldg(sb + h);
            const int32_t r = __ldg(A.g.rank + gid[h]);
            uint32_t *w = A.dom + off + (r >> 5);
            const uint32_t bit = 1u << (r & 31);
            if (w == dc.w && (dc.bits & bit)) continue;   // this lane set it already
            atomicOr(w, bit);   // no pre-check: these words miss L2, and a reduction does not wait
            if (w != dc.w) { dc.w = w; dc.bits = 0; }
            dc.bits |= bit;
        }
        return;
    }
    const int32_t P = __ldg(A.qp.pattern + slot);
    const uint64_t perm = __ldg(A.qp.perm + slot);
    {
        // PASS_EMIT
        const int32_t nid = __ldg(A.newid + P);
        if (nid < 0) return;
        const unsigned act = __activemask();
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(act) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(A.out_cursor, (unsigned long long)__popc(act));
        base = __shfl_sync(act, base, leader);
        const int64_t pos = (int64_t)base + __popc(act & ((1u << lane) - 1u));
        if (pos >= A.out_N) { atomicOr(A.err, FSM_ERR_BOUNDS); return; }
#pragma unroll
        for (int h = 0; h < K; ++h) A.out_v[(int64_t)nib_get(perm, h) * A.out_N + pos] = gid[h];
        A.out_pid[pos] = nid;
    }
}

// Edge-list quick pattern (the quick pattern of earlier systems that Section 6 compares the
// index-based one against): the joined subgraph's labels and edges listed with its vertices in
// ascending id order.  Bits 6h..6h+5 hold the label of the h-th smallest vertex; bit 42 + q holds
// pair q of (0,1), (0,2), ..., (K-2,K-1) over that order (K <= 7, so bit 63 stays clear and no
// key equals FSM_EMPTY_KEY).  sg receives the vertices in that order.
template <int K>
__device__ __forceinline__ uint64_t edge_list_key(const int32_t (&gid)[K], const int (&lab)[K], const uint32_t *adj,
                                                  int32_t (&sg)[K]) {
    int ord[K];
#pragma unroll
    for (int h = 0; h < K; ++h) ord[h] = h;
#pragma unroll
    for (int a = 1; a < K; ++a)
        for (int b = a; b > 0 && gid[ord[b - 1]] > gid[ord[b]]; --b) { const int t = ord[b]; ord[b] = ord[b - 1]; ord[b - 1] = t; }
    uint64_t key = 0;
    int bit = 42;
#pragma unroll
    for (int a = 0; a < K; ++a) {
        key |= (uint64_t)lab[ord[a]] << (6 * a);
        sg[a] = gid[ord[a]];
#pragma unroll
        for (int b = a + 1; b < K; ++b, ++bit)
            if ((adj[ord[a]] >> ord[b]) & 1u) key |= 1ull << bit;
    }
    return key;
}

// An accepted join under edge-list quick patterns: local position h is the h-th smallest vertex
// (sg), so domain and emission take their per-position data from sg directly.
template <int K, int PASS>
__device__ __forceinline__ void accept_sorted(const ExtArgs &A, CountCache *cc, uint64_t key, const int32_t (&sg)[K]) {
    if (PASS == PASS_COUNT) {
        const unsigned act = __activemask();
        const unsigned grp = __match_any_sync(act, key);
        const int lane = threadIdx.x & 31;
        if (lane == __ffs(grp) - 1) count_key(A, cc, key, __popc(grp));
        return;
    }
    const int64_t slot = qp_find(A.qp, key);
    if (slot < 0) { atomicOr(A.err, FSM_ERR_QP_MISSING); return; }
    if (PASS == PASS_DOMAIN) {
        const int64_t *sb = A.slot_base + slot * FSM_MAXK;
        if (__ldg(sb) < 0) return;
#pragma unroll
        for (int h = 0; h < K; ++h) {
            const int32_t r = __ldg(A.g.rank + sg[h]);
            uint32_t *w = A.dom + __ldg(sb + h) + (r >> 5);
            const uint32_t bit = 1u << (r & 31);
            if (!(__ldcg(w) & bit)) atomicOr(w, bit);
        }
        return;
    }
    if (PASS == PASS_EMIT) {
        const int32_t P = __ldg(A.qp.pattern + slot);
        const uint64_t perm = __ldg(A.qp.perm + slot);
        const int32_t nid = __ldg(A.newid + P);
        if (nid < 0) return;
        const unsigned long long pos = atomicAdd(A.out_cursor, 1ull);
        if ((int64_t)pos >= A.out_N) { atomicOr(A.err, FSM_ERR_BOUNDS); return; }
#pragma unroll
        for (int h = 0; h < K; ++h) A.out_v[(int64_t)nib_get(perm, h) * A.out_N + (int64_t)pos] = sg[h];
        A.out_pid[pos] = nid;
    }
}

// Join s (vertices S, pattern pid, key position i) with one piece.  Piece vertices pv[0..2]
// are in the piece's own order, pl their labels; shape is PIECE_WEDGE (centre pv[0]) or
// PIECE_TRI.
// Cross bits of a vertex x: bit p' set when x ~ s[p] (p != i, p' = p minus one if p > i),
// by binary search in the shorter neighbour list.
template <int L>
__device__ __forceinline__ uint32_t cross_bits(const ExtArgs &A, const int32_t (&S)[L], const int2 (&SR)[L], int i,
                                               int32_t x) {
    uint32_t c = 0;
    if constexpr (L >= 2) {
        const int32_t bx = __ldg(A.g.row_ptr + x), ex = __ldg(A.g.row_ptr + x + 1);
#pragma unroll
        for (int p = 0; p < L; ++p) {
            if (p == i) continue;
            const int pp = p < i ? p : p - 1;
            if (adj_rows(A.g.col, SR[p].x, SR[p].y, S[p], bx, ex, x)) c |= 1u << pp;
        }
    }
    return c;
}

// Join s (vertices S, pattern pid, key position i) with one piece.  Piece vertices pv[0..2]
// are in the piece's own order, pl their labels; shape is PIECE_WEDGE (centre pv[0]) or
// PIECE_TRI.  The piece's two non-key vertices are va and vb; their cross bits ca / cb are
// already known when have_a / have_b is set.
template <int L, int PASS, int V>
__device__ __forceinline__ void join_piece(const ExtArgs &A, const int32_t (&S)[L], const int (&SL)[L],
                                           const int2 (&SR)[L], uint64_t srows, int32_t pid, int i, int shape,
                                           const int32_t (&pv)[3], const int (&pl)[3], Tally &tl,
                                           CountCache *cc, DomCache &dc, int32_t va, uint32_t ca, bool have_a,
                                           uint32_t cb, bool have_b, const int32_t (&RK)[L]) {
    constexpr int K = L + 2;
    const uint32_t pidx = piece_index(shape, pl[0], pl[1], pl[2]);
    if (A.piece_freq && !__ldg(A.piece_freq + pidx)) return;
    if (A.piece_sel && !__ldg(A.piece_sel + pidx)) return;
    const int32_t v = S[i];
    const int jpos = pv[0] == v ? 0 : (pv[1] == v ? 1 : 2);
    const int q0 = jpos == 0 ? 1 : 0;
    const int q1 = jpos == 2 ? 1 : 2;
    const int32_t x0 = pv[q0], x1 = pv[q1];
    const int lx0 = pl[q0], lx1 = pl[q1];
    uint32_t tj0, tj1, txx;
    piece_join_edges(shape, jpos, tj0, tj1, txx);

    // cross adjacency between s \ {v} and {x0, x1}
    uint32_t avail = 0;
    if constexpr (L >= 2) {
        const bool x0a = x0 == va;
        const uint32_t c0 = x0a ? (have_a ? ca : cross_bits<L>(A, S, SR, i, x0))
                                : (have_b ? cb : cross_bits<L>(A, S, SR, i, x0));
        const uint32_t c1 = x0a ? (have_b ? cb : cross_bits<L>(A, S, SR, i, x1))
                                : (have_a ? ca : cross_bits<L>(A, S, SR, i, x1));
#pragma unroll
        for (int pp = 0; pp < L - 1; ++pp)
            avail |= ((c0 >> pp & 1u) << (2 * pp)) | ((c1 >> pp & 1u) << (2 * pp + 1));
    }
    const uint32_t srow_i = (uint32_t)(srows >> (8 * i)) & 0xffu;

    int32_t gid[K];
#pragma unroll
    for (int h = 0; h < L; ++h) gid[h] = S[h];
    gid[L] = x0;
    gid[L + 1] = x1;

    uint32_t sub = avail;
    for (;;) {
        ++tl.tested;
        bool keep = true;
        if (L >= 2 && A.piece_freq) {
            // joining-point pruning: every connected triple {v, s[p], t[q]} must be frequent
#pragma unroll
            for (int p = 0; p < L; ++p) {
                if (p == i) continue;
                const int pp = p < i ? p : p - 1;
                const uint32_t e1 = (srow_i >> p) & 1u;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const uint32_t e2 = q ? tj1 : tj0;
                    const uint32_t e3 = (sub >> (2 * pp + q)) & 1u;
                    if (e1 + e2 + e3 < 2) continue;
                    const int lx = q ? lx1 : lx0;
                    uint32_t idx;
                    if (e1 && e2 && e3) idx = tri_index(SL[i], SL[p], lx);
                    else if (e1 && e2) idx = wedge_index(SL[i], SL[p], lx);
                    else if (e1 && e3) idx = wedge_index(SL[p], SL[i], lx);
                    else idx = wedge_index(lx, SL[i], SL[p]);
                    if (!__ldg(A.piece_freq + idx)) keep = false;
                }
            }
        }
        uint32_t adjK[K];
        if (keep && (L >= 2 || V == FSM_EXPLORE_TV_EDGELIST)) join_graph(L, srows, i, tj0, tj1, txx, sub, adjK);
        if (keep && L >= 2) {
            // smallest-vertex-first dissection must return exactly (t, s)
            if constexpr (L == 2) {
                keep = dissect4_keeps(gid, adjK, i);
            } else {
                uint32_t lm = 0;
                int jn = -1;
                dissect3(K, gid, adjK, lm, jn);
                keep = (lm == ((1u << i) | (1u << L) | (1u << (L + 1)))) && jn == i;
            }
        }
        if (keep) {
            ++tl.accepted;
            if constexpr (V == FSM_EXPLORE_TV_EDGELIST) {
                int labK[K];
#pragma unroll
                for (int h = 0; h < L; ++h) labK[h] = SL[h];
                labK[L] = lx0;
                labK[L + 1] = lx1;
                int32_t sg[K];
                const uint64_t key = edge_list_key<K>(gid, labK, adjK, sg);
                accept_sorted<K, PASS>(A, cc, key, sg);
            } else {
                accept<L, K, PASS>(A, cc, dc, make_key((uint32_t)pid, pidx, i, jpos, sub, L), gid, RK);
            }
        }
        if (A.mode == 1 || sub == 0) break;
        sub = (sub - 1) & avail;
    }
}

// Cross bits of neighbour number x of the key vertex from the warp's masks (see extend_kernel).
template <int L>
__device__ __forceinline__ uint32_t mask_bits(const uint32_t *mk, int stride, int32_t x) {
    uint32_t c = 0;
#pragma unroll
    for (int pp = 0; pp < L - 1; ++pp) c |= ((mk[pp * stride + (x >> 5)] >> (x & 31)) & 1u) << pp;
    return c;
}

template <int L, int PASS, int V>
__device__ __forceinline__ void do_piece(const ExtArgs &A, const int32_t (&S)[L], const int (&SL)[L],
                                         const int2 (&SR)[L], uint64_t srows, int32_t pid, int i, int64_t lq, Tally &tl,
                                         CountCache *cc, DomCache &dc, const uint32_t *mk, int mstride,
                                         const int32_t (&RK)[L], int32_t cpos, int32_t &ecur, const ulonglong2 qab,
                                         uint64_t qc) {
    // quota draw: the j-th candidate run by this unit is candidate (a * j + b) mod c
    if (V == FSM_EXPLORE_TV_QUOTA && qc) lq = (int64_t)((qab.x * (uint64_t)lq + qab.y) % qc);
    const DevGraph &g = A.g;
    const int32_t v = S[i];
    const int32_t rp = __ldg(g.prow + v);               // the lists pieces are drawn from
    const int32_t d = __ldg(g.prow + v + 1) - rp;
    // centre pairs first: all pairs of v's list, or for l = 2 those with x < cpos
    const int64_t nt = L == 2 ? (int64_t)cpos * (cpos - 1) / 2 : (int64_t)d * (d - 1) / 2;
    const int64_t nc = L == 2 ? centre_pairs(d, cpos) : nt;
    // Decode the piece: a centre pair {a, b} of N(v), or an end piece v-a-b.  xa / xb are the
    // positions of a / b in v's list when known (for the shared-memory masks), -1 otherwise.
    const bool centre = lq < nc;
    int32_t a, b, xa, xb;
    if (centre) {
        int32_t y;
        if (lq < nt) {
            // pair (x < y) of the triangle y < cpos (all of the list when l != 2), lq = y(y-1)/2 + x
            y = (int32_t)((1.0f + sqrtf(1.0f + 8.0f * (float)lq)) * 0.5f);
            while ((int64_t)y * (y - 1) / 2 > lq) --y;
            while ((int64_t)(y + 1) * y / 2 <= lq) ++y;
            xa = (int32_t)(lq - (int64_t)y * (y - 1) / 2);
        } else {
            // l = 2, rows y >= cpos: cpos pairs each (32-bit division when it fits: a 64-bit
            // one is a long subroutine, and this runs once per pair)
            const int64_t r = lq - nt;
            if (r <= 0xffffffffll) {
                const uint32_t r32 = (uint32_t)r, c32 = (uint32_t)cpos, qd = r32 / c32;
                y = cpos + (int32_t)qd;
                xa = (int32_t)(r32 - qd * c32);
            } else {
                y = cpos + (int32_t)(r / cpos);
                xa = (int32_t)(r % cpos);
            }
        }
        xb = y;
        if (A.debug && (xa < 0 || xa >= y || y >= d)) { atomicOr(A.err, FSM_ERR_BOUNDS); return; }
        a = __ldg(g.pcol + rp + xa);
        b = __ldg(g.pcol + rp + y);
        if (L == 1 && a < v) return;                 // size-3 subgraphs keyed at their smallest vertex
    } else {
        const int64_t lq2 = lq - nc;
        // the end list holding lq2: largest lo with pend[lo] <= lq2.  A lane walks a unit's
        // pieces in increasing order, so it starts from its previous answer (ecur) and usually
        // stays there or moves one list on; otherwise it searches the rest of the range.
        int32_t lo = ecur;
        if (lo >= d || (int64_t)__ldg(g.pend + rp + lo) > lq2) lo = 0;
        if (lo + 1 < d && (int64_t)__ldg(g.pend + rp + lo + 1) <= lq2) {
            ++lo;
            if (lo + 1 < d && (int64_t)__ldg(g.pend + rp + lo + 1) <= lq2) {
                int32_t hi = d - 1;
                ++lo;
                while (lo < hi) {
                    const int32_t mid = (lo + hi + 1) >> 1;
                    if ((int64_t)__ldg(g.pend + rp + mid) <= lq2) lo = mid; else hi = mid - 1;
                }
            }
        }
        ecur = lo;
        xa = lo;
        xb = -1;
        if (A.debug && (lo < 0 || lo >= d)) { atomicOr(A.err, FSM_ERR_BOUNDS); return; }
        a = __ldg(g.pcol + rp + lo);
        if (A.debug) {
            const int64_t r = lq2 - __ldg(g.pend + rp + lo);
            if (a < 0 || a >= g.n || r < 0 || r >= (int64_t)(__ldg(g.prow + a + 1) - __ldg(g.prow + a))) {
                atomicOr(A.err, FSM_ERR_BOUNDS);
                return;
            }
        }
        b = __ldg(g.pcol + __ldg(g.prow + a) + (int32_t)(lq2 - __ldg(g.pend + rp + lo)));
        if (b == v) return;
        if (L == 1 && (a < v || b < v)) return;
    }
    if (in_s<L>(S, a) || in_s<L>(S, b)) return;
    if constexpr (L == 2) {
        // Four-vertex joins with w = S[1 - i]: the greedy dissection from the smallest vertex m
        // always succeeds (the one vertex left is adjacent to the 3-set), so the join survives
        // only if m is in the piece and m's first greedy step stays in it.  For a centre piece
        // (v next to a and b) that fails exactly when w < min(a, b): either m = w, or m = v and
        // w, the smallest neighbour of v, is taken before a and b.  For an end piece (v next to
        // a only) it fails when w < min(v, a, b), or when v is that minimum and w < a.
        // The first case is already cut from the centre pairs' index space (x < cpos).
        const int32_t w = S[1 - i];
        if (!centre) {
            const int32_t m = min(v, min(a, b));
            if (w < m || (m == v && w < a)) return;
        }
    }
    // closed triple: a centre pair with a ~ b (an end piece's b ~ v closes it as well, but that
    // triangle is the centre pair {a, b} of v and is joined from there)
    bool tri = false;
    if (centre) {
        const int64_t moff = g.tri_off ? __ldg(g.tri_off + v) : -1;
        if (moff >= 0)   // v's neighbour matrix: bit (xa, xb), xa < xb
            tri = (__ldg(g.tri_bits + moff + (int64_t)xa * ((d + 31) >> 5) + (xb >> 5)) >> (xb & 31)) & 1u;
        else
            tri = is_adj(g, a, b);
    }
    else if (A.mode == 1 && is_adj(g, v, b)) return;   // vertex-induced: only the triangle
    const int la = __ldg(g.labels + a), lb = __ldg(g.labels + b);
    const bool hm = mk != nullptr;
    const uint32_t ca = hm ? mask_bits<L>(mk, mstride, xa) : 0u;
    const uint32_t cb = hm && centre ? mask_bits<L>(mk, mstride, xb) : 0u;
    const bool have_b = hm && centre;
    // One call site of join_piece (it is large): the wedge (edge-induced, or an open triple)
    // and then the triangle of a closed centre pair.
    const int j0 = (centre && tri && A.mode == 1) ? 1 : 0;
    const int j1 = (centre && tri) ? 1 : 0;
#pragma unroll 1
    for (int jj = j0; jj <= j1; ++jj) {
        int32_t pv[3];
        int pl[3];
        int shape = PIECE_WEDGE;
        if (!centre) {
            pv[0] = a; pl[0] = la;
            if (lab_id_less(SL[i], v, lb, b)) { pv[1] = v; pl[1] = SL[i]; pv[2] = b; pl[2] = lb; }
            else { pv[1] = b; pl[1] = lb; pv[2] = v; pl[2] = SL[i]; }
        } else if (jj == 0) {
            pv[0] = v; pl[0] = SL[i];
            if (lab_id_less(la, a, lb, b)) { pv[1] = a; pl[1] = la; pv[2] = b; pl[2] = lb; }
            else { pv[1] = b; pl[1] = lb; pv[2] = a; pl[2] = la; }
        } else {
            shape = PIECE_TRI;
            int32_t t0 = v, t1 = a, t2 = b, tv;
            int m0 = SL[i], m1 = la, m2 = lb, tl_;
            if (lab_id_less(m1, t1, m0, t0)) { tv = t0; t0 = t1; t1 = tv; tl_ = m0; m0 = m1; m1 = tl_; }
            if (lab_id_less(m2, t2, m1, t1)) { tv = t1; t1 = t2; t2 = tv; tl_ = m1; m1 = m2; m2 = tl_; }
            if (lab_id_less(m1, t1, m0, t0)) { tv = t0; t0 = t1; t1 = tv; tl_ = m0; m0 = m1; m1 = tl_; }
            pv[0] = t0; pv[1] = t1; pv[2] = t2;
            pl[0] = m0; pl[1] = m1; pl[2] = m2;
        }
        join_piece<L, PASS, V>(A, S, SL, SR, srows, pid, i, shape, pv, pl, tl, cc, dc, a, ca, hm, cb, have_b, RK);
    }
}

// Single-vertex exploration (Section 6's ablation, l -> l+1): join s with one neighbour a of
// the key vertex v = s[i] (lq = a's position in v's list).  The new embedding s' = s + a holds
// the edge v-a and, edge-induced, any subset C of a's other edges into s (vertex-induced: all
// of them).  It is kept only when
//   (1) v is the smallest-id vertex of s that a is joined to in s', so one key position makes
//       it, and
//   (2) a is the largest-id vertex of s' whose removal leaves s' connected, so one parent makes
//       it: s' minus that vertex, which is connected and, by anti-monotonicity, frequent.
// Its quick pattern is <pid(s), label(a), i, C> (join code 3 marks the single-vertex form).
// There is no joining-point pruning: no size-3 table is computed in this mode.
template <int L, int PASS>
__device__ __forceinline__ void do_edge(const ExtArgs &A, const int32_t (&S)[L], const int2 (&SR)[L], uint64_t srows,
                                        int32_t pid, int i, int64_t lq, Tally &tl, CountCache *cc, DomCache &dc,
                                        const uint32_t *mk, int mstride, const int32_t (&RK)[L]) {
    constexpr int K = L + 1;
    const int32_t v = S[i];
    if (A.debug && (lq < 0 || lq >= __ldg(A.g.prow + v + 1) - __ldg(A.g.prow + v))) { atomicOr(A.err, FSM_ERR_BOUNDS); return; }
    const int32_t a = __ldg(A.g.pcol + __ldg(A.g.prow + v) + (int32_t)lq);
    if (in_s<L>(S, a)) return;
    uint32_t avail = 0;   // bit p' (p != i, p' = p minus one if p > i): a ~ s[p]
    if constexpr (L >= 2) avail = mk ? mask_bits<L>(mk, mstride, (int32_t)lq) : cross_bits<L>(A, S, SR, i, a);
    uint32_t above = 0;   // the same bits for the vertices of s with a larger id than v
#pragma unroll
    for (int p = 0; p < L; ++p)
        if (p != i && S[p] > v) above |= 1u << (p < i ? p : p - 1);
    if (A.mode == 1 && (avail & ~above)) return;   // vertex-induced: a smaller neighbour of a keys it
    const uint32_t cand = avail & above;
    const int la = __ldg(A.g.labels + a);
    int32_t gid[K];
#pragma unroll
    for (int h = 0; h < L; ++h) gid[h] = S[h];
    gid[L] = a;
    const uint32_t all = (1u << K) - 1u;
    uint32_t sub = cand;
    for (;;) {
        ++tl.tested;
        uint32_t adjK[K];
#pragma unroll
        for (int h = 0; h < L; ++h) adjK[h] = (uint32_t)(srows >> (8 * h)) & 0xffu;
        adjK[L] = 1u << i;
        adjK[i] |= 1u << L;
#pragma unroll
        for (int p = 0; p < L; ++p) {
            if (p == i || !((sub >> (p < i ? p : p - 1)) & 1u)) continue;
            adjK[p] |= 1u << L;
            adjK[L] |= 1u << p;
        }
        bool keep = true;
#pragma unroll
        for (int h = 0; h < L; ++h)
            if (keep && S[h] > a && mask_connected(all & ~(1u << h), adjK, K)) keep = false;
        if (keep) {
            ++tl.accepted;
            accept<L, K, PASS>(A, cc, dc, make_key((uint32_t)pid, (uint32_t)la, i, 3, sub, L), gid, RK);
        }
        if (A.mode == 1 || sub == 0) break;
        sub = (sub - 1) & cand;
    }
}

// Resident blocks per SM asked of the compiler.  The kernel is bound by load latency, so
// occupancy is bought with registers (what spills stays in L1).
#define FSM_EXT_MINB_COUNT 4
#define FSM_EXT_MINB_DOMAIN 4
template <int PASS> struct ExtMinBlocks {
    static constexpr int value = PASS == PASS_DOMAIN ? FSM_EXT_MINB_DOMAIN : FSM_EXT_MINB_COUNT;
};

template <int L, int PASS, int V = FSM_EXPLORE_TV>
__global__ void __launch_bounds__(256, ExtMinBlocks<PASS>::value) extend_kernel(ExtArgs A) {
    const int lane = threadIdx.x & 31;
    const int64_t nunits = A.ne * L;
    Tally tl{0ull, 0ull};
    DomCache dc;
    dc.w = nullptr;
    dc.bits = 0u;
    __shared__ uint32_t mask_s[8 * (L > 1 ? L - 1 : 1) * FSM_MASK_WORDS];   // per warp, see below
    extern __shared__ unsigned long long dyn_smem[];   // CountCache in PASS_COUNT launches
    constexpr bool counts = PASS == PASS_COUNT || PASS == PASS_FUSED;
    CountCache *cc = counts ? reinterpret_cast<CountCache *>(dyn_smem) : nullptr;
    if (counts) {
        for (int x = threadIdx.x; x < 8 * FSM_WARP_SLOTS; x += blockDim.x) {
            cc->key[x / FSM_WARP_SLOTS][x % FSM_WARP_SLOTS] = FSM_EMPTY_KEY;
            cc->cnt[x / FSM_WARP_SLOTS][x % FSM_WARP_SLOTS] = 0ull;
            if (PASS == PASS_FUSED) cc->slot[x / FSM_WARP_SLOTS][x % FSM_WARP_SLOTS] = -1;
        }
        __syncthreads();
    }
    int64_t total = A.total, nchunks = A.nchunks, chunk = A.chunk;
    if (total < 0) {
        // device-resident size: no host round trip between the prefix sum and this launch
        total = __ldg(A.unit_base + nunits);
        if (chunk <= 0) {
            // at least 64 chunks per warp, and at most about 16 units' pieces per chunk (a chunk
            // over at most 32 small units builds their cross masks)
            const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
            const int64_t per_unit = total / (nunits > 0 ? nunits : 1);
            chunk = 256;
            while (chunk < 16384 && total / chunk > warps * 64 && chunk * 2 <= 16 * per_unit) chunk <<= 1;
        }
        nchunks = (total + chunk - 1) / chunk;
    }
    if (A.stats && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(A.stats + 2, (unsigned long long)total);
    for (;;) {
        unsigned long long c = 0;
        if (lane == 0) {
            // stop early when the call ran out of time, when an overflowing count pass is to be
            // repeated with a larger table, or when a one-pass level is to be redone in two passes
            const int ew = *(volatile int *)A.err;
            bool stop = (ew & FSM_ERR_TIMEOUT) || (PASS == PASS_COUNT && (ew & FSM_ERR_QP_OVERFLOW)) ||
                        (PASS == PASS_FUSED && ew);
            if (!stop && A.time_limit_ns && global_ns() - __ldcg(A.time_start) > A.time_limit_ns) {
                atomicOr(A.err, FSM_ERR_TIMEOUT);
                stop = true;
            }
            c = stop ? ~0ull : atomicAdd(A.chunk_ctr, 1ull);
        }
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= (unsigned long long)nchunks) break;
        const int64_t q0 = (int64_t)c * chunk;
        const int64_t q1 = min(q0 + chunk, total);
        int64_t ulo = 0, uhi = 0;
        if (lane == 0) {
            ulo = last_le(A.unit_base, 0, nunits - 1, q0);
            uhi = last_le(A.unit_base, ulo, nunits - 1, q1 - 1);
        }
        ulo = __shfl_sync(0xffffffffu, ulo, 0);
        uhi = __shfl_sync(0xffffffffu, uhi, 0);
        // A chunk inside one unit (hub keys: most of the work) first records, for every
        // neighbour of the key vertex v, its adjacency to each other vertex of s as bit masks in
        // shared memory: the cross tests of centre pieces and of the first vertex of end pieces
        // then read a bit instead of searching a neighbour list.
        // Chunks across several units whose key vertices have at most 64 neighbours build the
        // same masks for each unit (two words per other position of s): a centre piece then
        // needs no search, an end piece one for its far vertex only.  Bit j of mvalid: unit
        // ulo + j has masks, at word j * 2 * (L - 1).
        const uint32_t *mk = nullptr;
        uint32_t mvalid = 0;
        if constexpr (L >= 2) {
            if (ulo != uhi && uhi - ulo < FSM_MASK_UNITS) {
                uint32_t *wm = mask_s + (threadIdx.x >> 5) * ((L - 1) * FSM_MASK_WORDS);
                const int nu = (int)(uhi - ulo) + 1;
                for (int j = 0; j < nu; ++j) {
                    const int64_t u = ulo + j;
                    const int64_t e = A.e0 + u / L;
                    const int iu = (int)(u % L);
                    const int32_t v = __ldg(A.fv + (int64_t)iu * A.fN + e);
                    const int32_t rb = __ldg(A.g.prow + v), dv = __ldg(A.g.prow + v + 1) - rb;
                    if (dv > 64) continue;
                    for (int p = 0; p < L; ++p) {
                        if (p == iu) continue;
                        const int pp = p < iu ? p : p - 1;
                        const int32_t sp = __ldg(A.fv + (int64_t)p * A.fN + e);
                        const int32_t sb = __ldg(A.g.row_ptr + sp), se = __ldg(A.g.row_ptr + sp + 1);
                        for (int32_t base = 0; base < dv; base += 32) {
                            bool bit = false;
                            if (base + lane < dv) {
                                const int32_t x = __ldg(A.g.pcol + rb + base + lane);
                                bit = adj_rows(A.g.col, sb, se, sp, __ldg(A.g.row_ptr + x), __ldg(A.g.row_ptr + x + 1), x);
                            }
                            const uint32_t word = __ballot_sync(0xffffffffu, bit);
                            if (lane == 0) wm[j * 2 * (L - 1) + pp * 2 + (base >> 5)] = word;
                        }
                    }
                    mvalid |= 1u << j;
                }
                __syncwarp();
            }
            if (ulo == uhi) {
                const int64_t e = A.e0 + ulo / L;
                const int iu = (int)(ulo % L);
                const int32_t v = __ldg(A.fv + (int64_t)iu * A.fN + e);
                const int32_t rb = __ldg(A.g.prow + v), dv = __ldg(A.g.prow + v + 1) - rb;
                if (dv <= FSM_MASK_WORDS * 32) {
                    uint32_t *wm = mask_s + (threadIdx.x >> 5) * ((L - 1) * FSM_MASK_WORDS);
#pragma unroll
                    for (int p = 0; p < L; ++p) {
                        if (p == iu) continue;
                        const int pp = p < iu ? p : p - 1;
                        const int32_t sp = __ldg(A.fv + (int64_t)p * A.fN + e);
                        const int32_t sb = __ldg(A.g.row_ptr + sp), se = __ldg(A.g.row_ptr + sp + 1);
                        for (int32_t base = 0; base < dv; base += 32) {
                            bool bit = false;
                            if (base + lane < dv) {
                                const int32_t x = __ldg(A.g.pcol + rb + base + lane);
                                bit = adj_rows(A.g.col, sb, se, sp, __ldg(A.g.row_ptr + x), __ldg(A.g.row_ptr + x + 1), x);
                            }
                            const uint32_t word = __ballot_sync(0xffffffffu, bit);
                            if (lane == 0) wm[pp * FSM_MASK_WORDS + (base >> 5)] = word;
                        }
                    }
                    __syncwarp();
                    mk = wm;
                }
            }
        }
        int64_t cur = -1, ub = 0;
        const uint32_t *lmk = mk;                       // this lane's unit's masks (or none)
        int lstride = FSM_MASK_WORDS;
        ulonglong2 qab = make_ulonglong2(0ull, 0ull);   // quota draw of the current unit
        uint64_t qc = 0;                                // its candidate count, 0 = no draw
        int32_t cpos = 0;   // l = 2: entries of the key vertex's list below the other vertex of s
        int32_t ecur = 0;   // end list of this lane's last end piece in the unit
        int32_t S[L];
        int SL[L];
        int2 SR[L];
        int32_t RK[L];
        int32_t pid = 0;
        int i = 0;
        uint64_t srows = 0;
        for (int64_t q = q0 + lane; q < q1; q += 32) {
            const int64_t u = (ulo == uhi) ? ulo : last_le(A.unit_base, ulo, uhi, q);
            if (u != cur) {
                cur = u;
                const int64_t e = A.e0 + u / L;
                i = (int)(u % L);
#pragma unroll
                for (int p = 0; p < L; ++p) {
                    S[p] = __ldg(A.fv + (int64_t)p * A.fN + e);
                    SL[p] = __ldg(A.g.labels + S[p]);
                    SR[p] = make_int2(__ldg(A.g.row_ptr + S[p]), __ldg(A.g.row_ptr + S[p] + 1));
                    RK[p] = (PASS == PASS_DOMAIN || PASS == PASS_FUSED) ? __ldg(A.g.rank + S[p]) : 0;
                }
                pid = __ldg(A.fpid + e);
                srows = L >= 2 ? __ldg(A.pat_adj + pid) : 0ull;
                ub = __ldg(A.unit_base + u);
                ecur = 0;
                if constexpr (L == 2 && V != FSM_EXPLORE_SV) {
                    const int32_t rb = __ldg(A.g.prow + S[i]);
                    cpos = count_below(A.g.pcol + rb, __ldg(A.g.prow + S[i] + 1) - rb, S[1 - i]);
                }
                if constexpr (V == FSM_EXPLORE_TV_QUOTA) {
                    // the unit's candidates before the quota cut (as the prefix kernel counted)
                    const int32_t v = S[i];
                    const int64_t d = __ldg(A.g.prow + v + 1) - __ldg(A.g.prow + v);
                    const int64_t pairs = d * (d - 1) / 2;
                    const int64_t c = (L == 2 ? centre_pairs(d, cpos) : pairs) + (__ldg(A.g.ppc + v) - pairs);
                    qc = 0;
                    if (A.quota > 0 && c > A.quota) {
                        uint64_t qa, qb;
                        quota_affine(quota_unit_hash(A.qseed, S, L, v), (uint64_t)c, qa, qb);
                        qab = make_ulonglong2(qa, qb);
                        qc = (uint64_t)c;
                    }
                }
#pragma unroll
                for (int p = 0; p < L; ++p) dc.soff[p] = -1;
                if (mvalid) {
                    const int j = (int)(u - ulo);
                    lmk = (mvalid >> j) & 1u ? mask_s + (threadIdx.x >> 5) * ((L - 1) * FSM_MASK_WORDS) + j * 2 * (L - 1)
                                             : nullptr;
                    lstride = 2;
                }
            }
            if constexpr (V == FSM_EXPLORE_SV)
                do_edge<L, PASS>(A, S, SR, srows, pid, i, q - ub, tl, cc, dc, lmk, lstride, RK);
            else
                do_piece<L, PASS, V>(A, S, SL, SR, srows, pid, i, q - ub, tl, cc, dc, lmk, lstride, RK, cpos, ecur, qab,
                                     qc);
        }
        if (counts) flush_warp_counts<PASS == PASS_FUSED>(A, cc);
    }

    // per-warp totals, one atomic per warp
    unsigned long long t0 = tl.tested, t1 = tl.accepted;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t0 += __shfl_xor_sync(0xffffffffu, t0, o);
        t1 += __shfl_xor_sync(0xffffffffu, t1, o);
    }
    if (lane == 0 && A.stats) {
        atomicAdd(A.stats + 0, t0);
        atomicAdd(A.stats + 1, t1);
    }
}

// Host launchers, one translation unit per pass.  V picks the exploration variant
// (FSM_EXPLORE_*); the fused pass exists for two-vertex exploration with index-based keys only.
cudaError_t launch_extend_count(int L, int V, const ExtArgs &A, int grid, cudaStream_t st);
cudaError_t launch_extend_domain(int L, int V, const ExtArgs &A, int grid, cudaStream_t st);
cudaError_t launch_extend_emit(int L, int V, const ExtArgs &A, int grid, cudaStream_t st);
cudaError_t launch_extend_fused(int L, const ExtArgs &A, int grid, cudaStream_t st);
cudaError_t occupancy_extend_fused(int L, int *blocks_per_sm);
cudaError_t occupancy_extend_count(int L, int V, int *blocks_per_sm);
cudaError_t occupancy_extend_domain(int L, int V, int *blocks_per_sm);
cudaError_t occupancy_extend_emit(int L, int V, int *blocks_per_sm);
// the variants' launchers (pass = PASS_COUNT, PASS_DOMAIN or PASS_EMIT)
cudaError_t launch_extend_sv(int pass, int L, const ExtArgs &A, int grid, cudaStream_t st);
cudaError_t occupancy_extend_sv(int pass, int L, int *blocks_per_sm);
cudaError_t launch_extend_edgelist(int pass, int L, const ExtArgs &A, int grid, cudaStream_t st);
cudaError_t occupancy_extend_edgelist(int pass, int L, int *blocks_per_sm);
cudaError_t launch_extend_quota(int pass, int L, const ExtArgs &A, int grid, cudaStream_t st);
cudaError_t occupancy_extend_quota(int pass, int L, int *blocks_per_sm);
// size 7 -> 9 (count and domain passes of the method's own form)
cudaError_t launch_extend_l7(int pass, const ExtArgs &A, int grid, cudaStream_t st);
cudaError_t occupancy_extend_l7(int pass, int *blocks_per_sm);

} // namespace fsm
