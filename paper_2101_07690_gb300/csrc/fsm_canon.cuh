// fsm_canon.cuh -- canonical codes of small labeled graphs on the device.
//
// The canonical code of a labeled K-vertex graph (K <= 9) is the lexicographically smallest
// (label sequence, adjacency sequence A(0,1), A(0,2), ..., A(K-2,K-1)) over all vertex orders
// (Section 4.4's isomorphism check, done once per distinct quick pattern).  The smallest label
// sequence is the sorted one, so only orders that keep each label's positions can be smallest.
// When there are few of those (at most FSM_ENUM_MAX) they are enumerated; otherwise (up to
// 9! = 362880 for an unlabeled 9-vertex graph) a depth-first search over ordered cells finds
// the minimum:
//   * positions are filled in order; the vertex at position c is taken from the cell that
//     holds position c (initially the cells are the label segments);
//   * once it is chosen, row c of the code (its adjacency to positions c+1..K-1) is smallest
//     when, inside every later cell, its non-neighbours come before its neighbours, so each
//     cell is split that way, which fixes row c;
//   * a branch whose code prefix is above the best complete code so far is cut, and of two
//     twins in one cell (same neighbours apart from each other; swapping them is an
//     automorphism fixing everything chosen) only the first is tried.
// Every order the search can complete is label-sorted and row-by-row minimal given the rows
// before, which is where the lexicographic minimum lies, and pruning only drops branches that
// cannot beat or differ from what is kept; so both ways give the same code.
#pragma once
#include "fsm_device.cuh"

#define FSM_ENUM_MAX 5040   // label-preserving orders enumerated directly (7!)

namespace fsm {

FSM_HD bool next_perm(int *a, int n) {
    int i = n - 2;
    while (i >= 0 && a[i] >= a[i + 1]) --i;
    if (i < 0) {
        for (int l = 0, r = n - 1; l < r; ++l, --r) { int t = a[l]; a[l] = a[r]; a[r] = t; }
        return false;
    }
    int j = n - 1;
    while (a[j] <= a[i]) --j;
    int t = a[i]; a[i] = a[j]; a[j] = t;
    for (int l = i + 1, r = n - 1; l < r; ++l, --r) { t = a[l]; a[l] = a[r]; a[r] = t; }
    return true;
}

// Advance perm to the next permutation that keeps every position's label (positions with equal
// labels form contiguous segments seg_start[c]..); false after the last one.
FSM_HD bool next_label_perm(int K, const int *seg_start, int *perm) {
    int c = K - 1;
    while (c >= 0) {
        const int s = seg_start[c];
        if (c - s + 1 >= 2 && next_perm(perm + s, c - s + 1)) return true;
        c = s - 1;
    }
    return false;
}

// Adjacency word of an order: pair (perm[c1], perm[c2]) of the order at bit np - 1 - q.
FSM_HD uint64_t adj_code(int K, const uint32_t *adj, const int *perm) {
    uint64_t code = 0;
    for (int c1 = 0; c1 < K; ++c1) {
        const uint32_t row = adj[perm[c1]];
        for (int c2 = c1 + 1; c2 < K; ++c2) code = (code << 1) | (uint64_t)((row >> perm[c2]) & 1u);
    }
    return code;
}

// Vertices sorted by (label, index) into perm; seg[c] = first position of c's label segment.
// Returns the number of label-preserving orders (product of the segments' factorials).
FSM_HD int64_t label_sort(int K, const int *lab, int *perm, int *seg) {
    for (int h = 0; h < K; ++h) perm[h] = h;
    for (int a = 1; a < K; ++a)          // insertion sort by label (stable)
        for (int b = a; b > 0 && lab[perm[b - 1]] > lab[perm[b]]; --b) { int t = perm[b]; perm[b] = perm[b - 1]; perm[b - 1] = t; }
    int64_t orders = 1;
    for (int c = 0; c < K; ++c) {
        seg[c] = (c > 0 && lab[perm[c]] == lab[perm[c - 1]]) ? seg[c - 1] : c;
        orders *= (int64_t)(c - seg[c] + 1);
    }
    return orders;
}

// The depth-first search of the header.  lab / adj: the graph; first >= 0 forces that vertex to
// position 0 (the graph with that vertex marked by a label of its own below all others).  Returns
// the smallest adjacency code; best[c] = the vertex at position c of one order attaining it.
static __host__ __device__ __noinline__ uint64_t canon_search(int K, const int *lab, const uint32_t *adj, int first,
                                                              int *best) {
    int ord[FSM_MAXK + 1][FSM_MAXK];   // per depth: the vertices by position, grouped in cells
    uint32_t bnd[FSM_MAXK + 1];        // per depth: bit p set when position p ends its cell
    uint32_t seen[FSM_MAXK + 1];       // per depth: vertices already taken up at that position
    uint32_t expd[FSM_MAXK + 1];       // per depth: those of them whose branch was searched
    uint64_t pre[FSM_MAXK + 1];        // per depth: the code rows above it
    const int np = K * (K - 1) / 2;
    {
        int n0 = 0;
        if (first >= 0) ord[0][n0++] = first;
        for (int h = 0; h < K; ++h)
            if (h != first) ord[0][n0++] = h;
        const int s0 = first >= 0 ? 1 : 0;
        for (int a = s0 + 1; a < K; ++a)
            for (int b = a; b > s0 && lab[ord[0][b - 1]] > lab[ord[0][b]]; --b) {
                const int t = ord[0][b]; ord[0][b] = ord[0][b - 1]; ord[0][b - 1] = t;
            }
        bnd[0] = 1u << (K - 1);
        if (first >= 0) bnd[0] |= 1u;
        for (int p = s0; p + 1 < K; ++p)
            if (lab[ord[0][p]] != lab[ord[0][p + 1]]) bnd[0] |= 1u << p;
    }
    seen[0] = expd[0] = 0;
    pre[0] = 0;
    bool have = false;
    uint64_t bc = 0;
    int c = 0;
    for (;;) {
        if (c >= K - 1) {
            // every row is known (the last position is what is left)
            if (!have || pre[c] < bc) {
                bc = pre[c];
                have = true;
                for (int p = 0; p < K; ++p) best[p] = ord[c][p];
            }
            if (c == 0) break;
            --c;
            continue;
        }
        int e = c;
        while (!((bnd[c] >> e) & 1u)) ++e;
        // next candidate for position c: not taken up yet, and no twin of a searched one (twins
        // of twins need not be twins, so only searched vertices are compared)
        int x = -1;
        for (int y = c; y <= e && x < 0; ++y) {
            const int w = ord[c][y];
            if ((seen[c] >> w) & 1u) continue;
            seen[c] |= 1u << w;
            bool twin = false;
            for (int w2 = 0; w2 < K && !twin; ++w2)
                if (((expd[c] >> w2) & 1u) && (adj[w] & ~(1u << w2)) == (adj[w2] & ~(1u << w))) twin = true;
            if (!twin) x = y;
        }
        if (x < 0) {
            if (c == 0) break;
            --c;
            continue;
        }
        const int w = ord[c][x];
        expd[c] |= 1u << w;
        int *o = ord[c + 1];
        for (int p = 0; p < K; ++p) o[p] = ord[c][p];
        o[x] = o[c];
        o[c] = w;
        uint32_t nb = bnd[c] | (1u << c);
        // split every later cell: non-neighbours of w first; row c follows
        uint64_t row = 0;
        for (int a = c + 1; a < K;) {
            int b = a;
            while (!((nb >> b) & 1u)) ++b;
            int tmp[FSM_MAXK], n0 = 0;
            for (int p = a; p <= b; ++p)
                if (!((adj[w] >> o[p]) & 1u)) tmp[n0++] = o[p];
            const int nn = n0;
            for (int p = a; p <= b; ++p)
                if ((adj[w] >> o[p]) & 1u) tmp[n0++] = o[p];
            for (int p = a; p <= b; ++p) {
                o[p] = tmp[p - a];
                row = (row << 1) | (uint64_t)(p - a >= nn ? 1u : 0u);
            }
            if (nn > 0 && nn <= b - a) nb |= 1u << (a + nn - 1);
            a = b + 1;
        }
        const int len = K - 1 - c;
        const uint64_t prefix = (pre[c] << len) | row;
        const int used = np - (K - 1 - c) * (K - 2 - c) / 2;   // bits in rows 0..c
        if (have && prefix > (bc >> (np - used))) continue;    // cannot reach the best: next candidate
        bnd[c + 1] = nb;
        pre[c + 1] = prefix;
        seen[c + 1] = expd[c + 1] = 0;
        ++c;
    }
    return bc;
}

// Label word and vertex order (4 bits per vertex) of the optimal order best[] (vertex at each
// canonical position).
FSM_HD void canon_words(int K, const int *lab, const int *best, unsigned long long &clab, uint64_t &inv) {
    unsigned long long l = 0;
    uint64_t iv = 0;
    for (int c = 0; c < K; ++c) {
        l |= clab_put(c, lab[best[c]]);
        iv |= nib_put(best[c], c);
    }
    clab = l;
    inv = iv;
}

// The canonical code by enumerating the label-preserving orders: what canonicalise does when
// there are at most FSM_ENUM_MAX of them (always for K <= 7).
static __host__ __device__ __noinline__ void canonicalise_enum(int K, const int *lab, const uint32_t *adj,
                                                               unsigned long long &clab, uint64_t &cadj, uint64_t &inv) {
    int perm[FSM_MAXK], seg[FSM_MAXK], best[FSM_MAXK];
    label_sort(K, lab, perm, seg);
    // within each segment start from ascending vertex index (next_perm enumerates from there)
    for (int c = 0; c < K; ++c)
        for (int b = c; b > seg[c] && perm[b - 1] > perm[b]; --b) { int t = perm[b]; perm[b] = perm[b - 1]; perm[b - 1] = t; }
    uint64_t bc = ~0ull;
    do {
        const uint64_t code = adj_code(K, adj, perm);
        if (code < bc) {
            bc = code;
            for (int c = 0; c < K; ++c) best[c] = perm[c];
        }
    } while (next_label_perm(K, seg, perm));
    cadj = bc;
    canon_words(K, lab, best, clab, inv);
}

// Canonical code of a labeled K-vertex graph: the smallest (label sequence, adjacency
// sequence) over all vertex orders.  clab: label word; cadj: adjacency word; inv: vertex h ->
// canonical position (4 bits each) in one optimal order.
static __host__ __device__ __noinline__ void canonicalise(int K, const int *lab, const uint32_t *adj,
                                                          unsigned long long &clab, uint64_t &cadj, uint64_t &inv) {
    int perm[FSM_MAXK], seg[FSM_MAXK], best[FSM_MAXK];
    if (label_sort(K, lab, perm, seg) <= FSM_ENUM_MAX) {
        canonicalise_enum(K, lab, adj, clab, cadj, inv);
        return;
    }
    cadj = canon_search(K, lab, adj, -1, best);
    canon_words(K, lab, best, clab, inv);
}

// The labeled graph a quick-pattern key denotes, in the key's local vertex order (the order the
// extension kernel's accept step uses for that key's positions).
static __host__ __device__ __noinline__ void key_graph(int V, int L, uint64_t key, const uint64_t *pat_lab8,
                                                       const uint64_t *pat_adj8, int &K, int *labH, uint32_t *adjH) {
    if (V == FSM_EXPLORE_TV_EDGELIST) {
        // labels and edges listed over the vertices in ascending id order
        K = L + 2;
        int bit = 42;
        for (int a = 0; a < K; ++a) adjH[a] = 0;
        for (int a = 0; a < K; ++a) {
            labH[a] = (int)(key >> (6 * a)) & 63;
            for (int b = a + 1; b < K; ++b, ++bit)
                if ((key >> bit) & 1ull) { adjH[a] |= 1u << b; adjH[b] |= 1u << a; }
        }
        return;
    }
    uint32_t pid, pidx, cross;
    int i, jpos;
    split_key(key, L, pid, pidx, i, jpos, cross);
    const uint64_t lab8 = pat_lab8[pid], srows = pat_adj8[pid];
    for (int h = 0; h < L; ++h) labH[h] = (int)(lab8 >> (8 * h)) & 0xff;
    if (V == FSM_EXPLORE_SV) {
        // <pid(s), label(a), i, cross bits>: a joined to s[i] and to the cross positions
        K = L + 1;
        for (int h = 0; h < L; ++h) adjH[h] = (uint32_t)(srows >> (8 * h)) & 0xffu;
        labH[L] = (int)(pidx & 63);
        adjH[L] = 1u << i;
        adjH[i] |= 1u << L;
        for (int p = 0; p < L; ++p) {
            if (p == i || !((cross >> (p < i ? p : p - 1)) & 1u)) continue;
            adjH[p] |= 1u << L;
            adjH[L] |= 1u << p;
        }
        return;
    }
    K = L + 2;
    const int shape = (int)(pidx >> 18);
    const int pl[3] = {(int)(pidx >> 12) & 63, (int)(pidx >> 6) & 63, (int)pidx & 63};
    const int q0 = jpos == 0 ? 1 : 0;
    const int q1 = jpos == 2 ? 1 : 2;
    labH[L] = pl[q0];
    labH[L + 1] = pl[q1];
    uint32_t tj0, tj1, txx;
    piece_join_edges(shape, jpos, tj0, tj1, txx);
    join_graph(L, srows, i, tj0, tj1, txx, cross, adjH);
}

FSM_HD void decode_code(int K, unsigned long long clab, uint64_t cadj, int *lab, uint32_t *adj) {
    const int np = K * (K - 1) / 2;
    for (int c = 0; c < K; ++c) { lab[c] = clab_get(clab, c); adj[c] = 0; }
    int q = 0;
    for (int c1 = 0; c1 < K; ++c1)
        for (int c2 = c1 + 1; c2 < K; ++c2, ++q)
            if ((cadj >> (np - 1 - q)) & 1ull) { adj[c1] |= 1u << c2; adj[c2] |= 1u << c1; }
}


// Orbit representatives by marking: c and c' (of one label) share an orbit exactly when the
// graph with c marked and the graph with c' marked have the same canonical code.  seg[c] = the
// first position of c's label segment.
static __host__ __device__ __noinline__ void orbit_reps_search(int K, const int *lab, const uint32_t *adj,
                                                               const int *seg, int *rep) {
    uint64_t mark[FSM_MAXK];
    int tmp[FSM_MAXK];
    for (int c = 0; c < K; ++c) {
        rep[c] = c;
        mark[c] = canon_search(K, lab, adj, c, tmp);
        for (int c2 = seg[c]; c2 < c; ++c2)
            if (rep[c2] == c2 && mark[c2] == mark[c]) { rep[c] = c2; break; }
    }
}

// Orbit representatives of a canonical pattern: rep[c] = the smallest canonical position that
// an automorphism (a label-preserving order with the same adjacency sequence) maps c to.  With
// few label-preserving orders they are enumerated (orbit_reps_enum), otherwise found by
// marking.
static __host__ __device__ __noinline__ void orbit_reps_enum(int K, unsigned long long clab, uint64_t cadj, int *rep) {
    int lab[FSM_MAXK], perm[FSM_MAXK], seg[FSM_MAXK];
    uint32_t adj[FSM_MAXK];
    decode_code(K, clab, cadj, lab, adj);
    for (int c = 0; c < K; ++c) {
        perm[c] = c;
        rep[c] = c;
        seg[c] = (c > 0 && lab[c] == lab[c - 1]) ? seg[c - 1] : c;
    }
    do {
        if (adj_code(K, adj, perm) == cadj)
            for (int c = 0; c < K; ++c) if (perm[c] < rep[c]) rep[c] = perm[c];
    } while (next_label_perm(K, seg, perm));
}

static __host__ __device__ __noinline__ void orbit_reps(int K, unsigned long long clab, uint64_t cadj, int *rep) {
    int lab[FSM_MAXK], seg[FSM_MAXK];
    uint32_t adj[FSM_MAXK];
    decode_code(K, clab, cadj, lab, adj);
    int64_t orders = 1;
    for (int c = 0; c < K; ++c) {
        seg[c] = (c > 0 && lab[c] == lab[c - 1]) ? seg[c - 1] : c;
        orders *= (int64_t)(c - seg[c] + 1);
    }
    if (orders <= FSM_ENUM_MAX) {
        orbit_reps_enum(K, clab, cadj, rep);
        return;
    }
    orbit_reps_search(K, lab, adj, seg, rep);
}

// A canonical code of K <= 7 vertices in 63 bits: label of canonical position c at bits
// 6c..6c+5, the adjacency sequence (as canonicalise returns it) from bit 42.  Bit 63 stays clear,
// so no packed code equals FSM_EMPTY_KEY.
FSM_HD uint64_t pack_code(int K, unsigned long long clab, uint64_t cadj) {
    uint64_t k = 0;
    for (int c = 0; c < K; ++c) k |= (uint64_t)clab_get(clab, c) << (6 * c);
    return k | (cadj << 42);
}

} // namespace fsm
