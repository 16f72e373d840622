// fsm_device.cuh -- device-side building blocks shared by the mining kernels.
//
// Vocabulary (paper Sections 3-4):
//   embedding  a connected size-l subgraph of G, stored as l vertex ids in the canonical order
//              of its pattern plus the pattern id (Section 4.4 stores pattern_idx with each
//              embedding);
//   piece      a connected size-3 subgraph (wedge or triangle) that the size-l embedding is
//              joined with on one shared vertex (two-vertex exploration, Section 4.1);
//   key        the joining vertex v = s[i] (Section 4.2 groups subgraphs by column vertex);
//   cross edge an edge between s \ {v} and t \ {v}; edge-induced joins enumerate every subset
//              of the existing cross edges, vertex-induced joins take all of them (Section 4.1);
//   QP         index-based quick pattern <pid(s), pid(t), join positions, cross bit array>
//              (Section 4.4).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define FSM_MAXK 9
#define FSM_MAXL 7               // largest stored level that is still extended (k <= 9)

// exploration variants of the extension kernel (option "explore" and "quick_pattern")
#define FSM_EXPLORE_TV 0           // two-vertex exploration, index-based quick patterns (the method)
#define FSM_EXPLORE_SV 1           // single-vertex exploration (l -> l+1), index-based quick patterns
#define FSM_EXPLORE_TV_EDGELIST 2  // two-vertex exploration, edge-list quick patterns
#define FSM_EXPLORE_TV_QUOTA 3     // two-vertex exploration with per-key-group sampling quotas
#define FSM_EMPTY_KEY 0xFFFFFFFFFFFFFFFFull
#define FSM_HD __host__ __device__ __forceinline__

// error bits written by kernels into the per-call error word
#define FSM_ERR_QP_OVERFLOW  1   // quick-pattern table too full: grow and repeat the pass
#define FSM_ERR_QP_MISSING   2   // a key seen in a later pass was not in the table
#define FSM_ERR_BOUNDS       4   // an index check failed
#define FSM_ERR_CSR          8   // malformed CSR found by validation
#define FSM_ERR_POOL        16   // the one-pass last level ran out of bitmap pool: two passes instead
#define FSM_ERR_CODE_FULL   32   // the one-pass last level's pattern table is full: two passes instead
#define FSM_ERR_TIMEOUT     64   // the call's time limit ran out (option "time_limit_ms")

namespace fsm {

// ---------------------------------------------------------------------------- graph

struct DevGraph {
    int32_t n;
    int64_t nnz;
    const int32_t *row_ptr;   // [n+1]
    const int32_t *col;       // [nnz], rows sorted ascending
    const int32_t *labels;    // [n]
    const int32_t *rank;      // [n] index of v within its label class
    const int64_t *piece_cnt; // [n] piece slots keyed at v: C(d,2) + sum_{a in N(v)} d(a)
    const int32_t *end_off;   // [nnz] exclusive prefix of d(a) over N(v), per row
    // Lists the pieces are drawn from.  Exact mining: the graph itself (prow = row_ptr, ...).
    // Sampled last level: the kept directed edges only (piece_cnt / end_off computed on them);
    // adjacency tests always use row_ptr / col.
    const int32_t *prow, *pcol, *pend;
    const int64_t *ppc;
    // Neighbour adjacency of high-degree vertices: for v with tri_off[v] >= 0, bit y of row x
    // (x < y < d(v)) of a d(v) x ceil(d(v)/32)-word matrix at word tri_off[v] of tri_bits says
    // whether the x-th and y-th neighbours of v are adjacent.  Indexed by positions in the
    // graph's own lists, so it is NULL while pieces come from other lists (sampled level).
    const int64_t *tri_off;
    const uint32_t *tri_bits;
};

// Is w a neighbour of u?  Binary search in the shorter of the two sorted lists.
__device__ __forceinline__ bool is_adj(const DevGraph &g, int32_t u, int32_t w) {
    int32_t bu = __ldg(g.row_ptr + u), eu = __ldg(g.row_ptr + u + 1);
    int32_t bw = __ldg(g.row_ptr + w), ew = __ldg(g.row_ptr + w + 1);
    int32_t lo, end, x;
    if (eu - bu <= ew - bw) { lo = bu; end = eu; x = w; } else { lo = bw; end = ew; x = u; }
    int32_t hi = end;
    while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        int32_t c = __ldg(g.col + mid);
        if (c < x) lo = mid + 1; else hi = mid;
    }
    return lo < end && __ldg(g.col + lo) == x;
}

// ---------------------------------------------------------------------------- pieces
//
// A piece's own order (used only inside quick-pattern keys): wedge = [centre, end, end],
// ends ordered by (label, id); triangle = its three vertices ordered by (label, id).  Any
// order that realises the piece's shape and label sequence keeps the quick pattern sound.
// Piece index: shape bit (1 = triangle) << 18 | label0 << 12 | label1 << 6 | label2.

enum { PIECE_WEDGE = 0, PIECE_TRI = 1 };
#define FSM_PIECE_SPACE (1 << 19)

// Entries of the sorted list a[0, n) below x.
FSM_HD int32_t count_below(const int32_t *a, int32_t n, int32_t x) {
    int32_t lo = 0, hi = n;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Centre pairs a unit enumerates.  In general every pair x < y of the key vertex's list of
// length d.  When s is one edge {v, w} (l = 2), the join survives dissection only if the piece
// holds a vertex below w (see do_piece), so only pairs whose smaller end a (position x) is below
// w are enumerated: x < c, c = entries of v's list below w.  Rows y < c hold y pairs, later rows
// c pairs each.
FSM_HD int64_t centre_pairs(int64_t d, int64_t c) {
    return c * (c - 1) / 2 + (d - c) * c;
}

FSM_HD uint32_t piece_index(int shape, int l0, int l1, int l2) {
    return ((uint32_t)shape << 18) | ((uint32_t)l0 << 12) | ((uint32_t)l1 << 6) | (uint32_t)l2;
}

FSM_HD bool lab_id_less(int la, int32_t ia, int lb, int32_t ib) {
    return la < lb || (la == lb && ia < ib);
}

// Index of the size-3 pattern formed by a wedge with centre label c and end labels x, y.
FSM_HD uint32_t wedge_index(int c, int x, int y) {
    return x <= y ? piece_index(PIECE_WEDGE, c, x, y) : piece_index(PIECE_WEDGE, c, y, x);
}
FSM_HD uint32_t tri_index(int x, int y, int z) {
    int a = x, b = y, c = z, t;
    if (a > b) { t = a; a = b; b = t; }
    if (b > c) { t = b; b = c; c = t; }
    if (a > b) { t = a; a = b; b = t; }
    return piece_index(PIECE_TRI, a, b, c);
}

// ---------------------------------------------------------------------------- QP keys
//
// 64-bit key of a join from a size-l embedding: pid_s (24 bits) | piece index (19) | i (3) |
// j (2) | cross bits (2*(l-1)).  Cross bit (p', q): s position p (p' = p minus one if p > i)
// adjacent to the piece's q-th non-joining vertex, bit index p' * 2 + q.  Up to l = 6 the cross
// field has 10 bits; from l = 7 it has 12 and every other field sits two bits higher
// (key_shift).  The top bits stay clear, so no key equals FSM_EMPTY_KEY.

#define FSM_PID_BITS 24
FSM_HD int key_shift(int L) { return L >= 7 ? 2 : 0; }
FSM_HD uint64_t make_key(uint32_t pid_s, uint32_t pidx, int i, int j, uint32_t cross, int L) {
    const int w = key_shift(L);
    return ((uint64_t)pid_s << (34 + w)) | ((uint64_t)pidx << (15 + w)) | ((uint64_t)i << (12 + w)) |
           ((uint64_t)j << (10 + w)) | (uint64_t)cross;
}
FSM_HD void split_key(uint64_t key, int L, uint32_t &pid_s, uint32_t &pidx, int &i, int &j, uint32_t &cross) {
    const int w = key_shift(L);
    pid_s = (uint32_t)(key >> (34 + w)) & ((1u << FSM_PID_BITS) - 1);
    pidx = (uint32_t)(key >> (15 + w)) & ((1u << 19) - 1);
    i = (int)(key >> (12 + w)) & 7;
    j = (int)(key >> (10 + w)) & 3;
    cross = (uint32_t)key & ((1u << (10 + w)) - 1u);
}

// ---------------------------------------------------------------------------- pattern words
//
// A pattern of K <= 9 vertices in canonical order is held as
//   a label word: the label of canonical position c (6 bits; labels are below 64) at bits
//     6 (8 - c) .. 6 (8 - c) + 5, so that integer order is label-sequence order;
//   an adjacency word: the adjacency sequence A(0,1), A(0,2), ..., A(K-2,K-1), first pair most
//     significant (at most 36 bits), so that integer order is sequence order;
//   an orbit word: the orbit representative of canonical position c at bits 4c .. 4c + 3;
// and a vertex order (local vertex h -> canonical position) as 4 bits per vertex, at 4h.

FSM_HD int clab_get(unsigned long long clab, int c) { return (int)(clab >> (6 * (FSM_MAXK - 1 - c))) & 63; }
FSM_HD unsigned long long clab_put(int c, int lab) {
    return (unsigned long long)(lab & 63) << (6 * (FSM_MAXK - 1 - c));
}
FSM_HD int nib_get(uint64_t w, int h) { return (int)(w >> (4 * h)) & 15; }
FSM_HD uint64_t nib_put(int h, int v) { return (uint64_t)(v & 15) << (4 * h); }

FSM_HD uint64_t mix64(uint64_t x) {
    x ^= x >> 31; x *= 0x7fb5d329728ea185ull;
    x ^= x >> 27; x *= 0x81dadef4bc2dd44dull;
    x ^= x >> 33; return x;
}

// ---------------------------------------------------------------------------- sampling
//
// Sampled last level: the directed edge (x -> y) is kept iff H(H(H(seed) ^ x) ^ y) < thr,
// thr = floor(q * 2^64) with q = sqrt(p), where H is one step of splitmix64 (Steele, Lea,
// Flood, "Fast splittable pseudorandom number generators", 2014): add the golden gamma
// 0x9e3779b97f4a7c15, then the variant-13 mix.  A centre piece {v; a, b} is joined iff both
// v -> a and v -> b are kept, an end piece v - a - b iff v -> a and a -> b are kept, so about
// p of the pieces survive and only those are enumerated.

FSM_HD uint64_t splitmix_step(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

FSM_HD bool keep_edge(uint64_t seed, uint64_t thr, int32_t x, int32_t y) {
    uint64_t h = splitmix_step(seed);
    h = splitmix_step(h ^ (uint64_t)(uint32_t)x);
    h = splitmix_step(h ^ (uint64_t)(uint32_t)y);
    return h < thr;
}

// ---------------------------------------------------------------------------- sampling quotas
//
// Section 5's sampling with fixed iteration counts: a loop over the candidates of one key group
// runs all of them when there are at most Q, otherwise Q drawn uniformly.  Here a key group is
// one unit (stored embedding s, key vertex v = s[i]) and its loop runs over the unit's candidate
// pieces, numbered as the extension kernel enumerates them (centre pairs of v's list, then end
// pieces along v's list).  A unit with c > Q candidates runs candidates (a * j + b) mod c for
// j = 0 .. Q-1: a uniformly placed, randomly strided arithmetic progression, Q distinct pieces
// since gcd(a, c) = 1.  a and b come from the unit hash
//     h = H(... H(H(seed) ^ x_0) ... ^ x_{l-1}) then h = H(h ^ (2^32 + v))
// over the ids x_0 < ... < x_{l-1} of s (so the draw does not depend on the order in which s
// is stored), H one splitmix64 step: a = the first integer coprime to c at or after
// 1 + (h mod (c - 1)), wrapping from c - 1 to 1, and b = H(h) mod c.
// When an edge list is joined (l = 2), the edges of each key vertex v are sampled too: with
// d(v) > X, the unit of edge {v, w} runs only if (a_v * pos + b_v) mod d(v) < X, pos = w's
// position in v's list and (a_v, b_v) drawn as above from g_v = H(H(seed) ^ (2^33 + v)) and
// modulus d(v): X of v's edges, uniformly.

FSM_HD uint64_t gcd_u64(uint64_t x, uint64_t y) {
    while (y) {
        const uint64_t t = x % y;
        x = y;
        y = t;
    }
    return x;
}

// a, b of the affine draw for modulus c >= 2 from hash h
FSM_HD void quota_affine(uint64_t h, uint64_t c, uint64_t &a, uint64_t &b) {
    a = 1 + h % (c - 1);
    while (gcd_u64(a, c) != 1) a = a + 1 == c ? 1 : a + 1;
    b = splitmix_step(h) % c;
}

// unit hash of embedding s (ids in any order, L <= FSM_MAXL) joined at v
FSM_HD uint64_t quota_unit_hash(uint64_t seed, const int32_t *ids, int L, int32_t v) {
    int32_t s[FSM_MAXL];
    for (int h = 0; h < L; ++h) s[h] = ids[h];
    for (int a = 1; a < L; ++a)
        for (int b = a; b > 0 && s[b - 1] > s[b]; --b) { const int32_t t = s[b]; s[b] = s[b - 1]; s[b - 1] = t; }
    uint64_t h = splitmix_step(seed);
    for (int a = 0; a < L; ++a) h = splitmix_step(h ^ (uint64_t)(uint32_t)s[a]);
    return splitmix_step(h ^ ((1ull << 32) + (uint64_t)(uint32_t)v));
}

// Does the unit of edge {v, w} (w at position pos of v's list of length d) run under an edge
// quota X?
FSM_HD bool quota_edge_kept(uint64_t seed, int32_t v, int64_t pos, int64_t d, int64_t X) {
    if (d <= X) return true;
    uint64_t a, b;
    quota_affine(splitmix_step(splitmix_step(seed) ^ ((1ull << 33) + (uint64_t)(uint32_t)v)), (uint64_t)d, a, b);
    return (a * (uint64_t)pos + b) % (uint64_t)d < (uint64_t)X;
}

// ---------------------------------------------------------------------------- dissection
//
// Smallest-vertex-first dissection of a connected K-vertex subgraph into a 3-vertex part l and
// a (K-2)-vertex part r sharing one vertex (Algorithm 1, function dissect with n = 3): for each
// start vertex in ascending id order, span greedily (always adding the smallest unvisited
// vertex adjacent to the visited set) until 3 vertices are visited; the remaining vertices
// plus one visited vertex v' (tried in ascending id order) must be connected.  If no start
// vertex yields a dissection, the exhaustive rule below answers: the smallest (sorted ids of
// l, id of v') over every connected 3-set l with connected remainder.  Any total and
// deterministic rule keeps exactly one join per subgraph; the greedy rule is the paper's.

FSM_HD int popc32(uint32_t x) {
#ifdef __CUDA_ARCH__
    return __popc(x);
#else
    return __builtin_popcount(x);
#endif
}

FSM_HD bool mask_connected(uint32_t m, const uint32_t *adj, int K) {
    if (!m) return false;
    uint32_t seen = m & (0u - m), front = seen;
    while (front) {
        uint32_t nx = 0;
        for (int h = 0; h < K; ++h)
            if (front >> h & 1u) nx |= adj[h];
        nx &= m & ~seen;
        seen |= nx;
        front = nx;
    }
    return seen == m;
}

FSM_HD int smallest_in(uint32_t m, const int32_t *gid, int K) {
    int best = -1;
    for (int h = 0; h < K; ++h)
        if ((m >> h & 1u) && (best < 0 || gid[h] < gid[best])) best = h;
    return best;
}

// The exhaustive rule, out of line: it almost never runs, and keeping it out of the join path
// keeps that path small in the instruction cache.
static __host__ __device__ __noinline__ void dissect3_exhaustive(int K, const int32_t *gid, const uint32_t *adj,
                                                         uint32_t &l_mask, int &join) {
    const uint32_t all = (1u << K) - 1u;
    l_mask = 0; join = -1;
    int32_t bk0 = 0, bk1 = 0, bk2 = 0, bkv = 0;
    for (uint32_t m = 0; m <= all; ++m) {
        if (popc32(m) != 3 || !mask_connected(m, adj, K)) continue;
        int32_t ids[3]; int c = 0;
        for (int h = 0; h < K; ++h) if (m >> h & 1u) ids[c++] = gid[h];
        int32_t t;
        if (ids[0] > ids[1]) { t = ids[0]; ids[0] = ids[1]; ids[1] = t; }
        if (ids[1] > ids[2]) { t = ids[1]; ids[1] = ids[2]; ids[2] = t; }
        if (ids[0] > ids[1]) { t = ids[0]; ids[0] = ids[1]; ids[1] = t; }
        for (int h = 0; h < K; ++h) {
            if (!(m >> h & 1u)) continue;
            if (!mask_connected((all & ~m) | (1u << h), adj, K)) continue;
            bool better = l_mask == 0 ||
                ids[0] < bk0 || (ids[0] == bk0 && (ids[1] < bk1 || (ids[1] == bk1 &&
                (ids[2] < bk2 || (ids[2] == bk2 && gid[h] < bkv)))));
            if (better) { l_mask = m; join = h; bk0 = ids[0]; bk1 = ids[1]; bk2 = ids[2]; bkv = gid[h]; }
        }
    }
}

// Returns true when the greedy rule answered, false when the exhaustive rule did.
// l_mask = 0 means no dissection exists (the input was not connected).
FSM_HD bool dissect3(int K, const int32_t *gid, const uint32_t *adj, uint32_t &l_mask, int &join) {
    const uint32_t all = (1u << K) - 1u;
    uint32_t tried = 0;
    for (int it = 0; it < K; ++it) {
        int h0 = smallest_in(all & ~tried, gid, K);
        tried |= 1u << h0;
        uint32_t vis = 1u << h0;
        bool ok = true;
        for (int s = 0; s < 2; ++s) {
            uint32_t cand = 0;
            for (int h = 0; h < K; ++h)
                if (vis >> h & 1u) cand |= adj[h];
            cand &= all & ~vis;
            int hb = smallest_in(cand, gid, K);
            if (hb < 0) { ok = false; break; }
            vis |= 1u << hb;
        }
        if (!ok) continue;
        uint32_t rest = all & ~vis, rem = vis;
        while (rem) {
            int hv = smallest_in(rem, gid, K);
            rem &= ~(1u << hv);
            if (mask_connected(rest | (1u << hv), adj, K)) { l_mask = vis; join = hv; return true; }
        }
    }
    dissect3_exhaustive(K, gid, adj, l_mask, join);
    return false;
}

// ---------------------------------------------------------------------------- join graph
//
// The (l+2)-vertex graph of one join, in local numbering: h < l are the size-l embedding's
// canonical positions (rows from its pattern's adjacency bytes), h = l and l+1 are the piece's
// first and second non-joining vertices (piece order), joined to s[i] by the piece's edges and
// to s \ {s[i]} by the cross bits.  Both the extension kernel and the canonicalisation kernel
// build it with this function, so a quick-pattern key always denotes the graph that was
// dissected.

FSM_HD void piece_join_edges(int shape, int jpos, uint32_t &tj0, uint32_t &tj1, uint32_t &txx) {
    const int q0 = jpos == 0 ? 1 : 0;
    tj0 = (shape == PIECE_TRI || jpos == 0 || q0 == 0) ? 1u : 0u;   // always 1: a wedge's end sits next to its centre
    tj1 = (shape == PIECE_TRI || jpos == 0) ? 1u : 0u;
    txx = (shape == PIECE_TRI || q0 == 0) ? 1u : 0u;
}

FSM_HD void join_graph(int L, uint64_t srows, int i, uint32_t tj0, uint32_t tj1, uint32_t txx,
                       uint32_t cross, uint32_t *adjK) {
    for (int h = 0; h < L; ++h) adjK[h] = (uint32_t)(srows >> (8 * h)) & 0xffu;
    adjK[L] = 0;
    adjK[L + 1] = 0;
    if (tj0) { adjK[i] |= 1u << L; adjK[L] |= 1u << i; }
    if (tj1) { adjK[i] |= 1u << (L + 1); adjK[L + 1] |= 1u << i; }
    if (txx) { adjK[L] |= 1u << (L + 1); adjK[L + 1] |= 1u << L; }
    for (int p = 0; p < L; ++p) {
        if (p == i) continue;
        const int pp = p < i ? p : p - 1;
        if (cross >> (2 * pp) & 1u) { adjK[p] |= 1u << L; adjK[L] |= 1u << p; }
        if (cross >> (2 * pp + 1) & 1u) { adjK[p] |= 1u << (L + 1); adjK[L + 1] |= 1u << p; }
    }
}

} // namespace fsm
