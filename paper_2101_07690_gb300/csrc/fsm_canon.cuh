// fsm_canon.cuh -- canonical codes of small labeled graphs on the device.
//
// The canonical code of a labeled K-vertex graph (K <= 8) is the lexicographically smallest
// (label sequence, adjacency sequence A(0,1), A(0,2), ..., A(K-2,K-1)) over all vertex orders
// (Section 4.4's isomorphism check, done once per distinct quick pattern).  Only label-
// preserving orders of the label-sorted positions can be smallest, so only those are
// enumerated (at most 8! = 40320).
#pragma once
#include "fsm_device.cuh"

namespace fsm {

__device__ __forceinline__ bool next_perm(int *a, int n) {
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
__device__ __forceinline__ bool next_label_perm(int K, const int *seg_start, int *perm) {
    int c = K - 1;
    while (c >= 0) {
        const int s = seg_start[c];
        if (c - s + 1 >= 2 && next_perm(perm + s, c - s + 1)) return true;
        c = s - 1;
    }
    return false;
}

__device__ __forceinline__ uint32_t adj_code(int K, const uint32_t *adj, const int *perm) {
    uint32_t code = 0;
    for (int c1 = 0; c1 < K; ++c1) {
        const uint32_t row = adj[perm[c1]];
        for (int c2 = c1 + 1; c2 < K; ++c2) code = (code << 1) | ((row >> perm[c2]) & 1u);
    }
    return code;
}

// Canonical code of a labeled K-vertex graph: the smallest (label sequence, adjacency
// sequence) over all vertex orders.  The smallest label sequence is the sorted one, so only
// label-preserving orders of the sorted positions are enumerated.  inv[h] = canonical
// position of vertex h in the first optimal order.
static __device__ __noinline__ void canonicalise(int K, const int *lab, const uint32_t *adj, unsigned long long &clab,
                             uint32_t &cadj, uint32_t &inv) {
    int perm[FSM_MAXK], seg[FSM_MAXK], best[FSM_MAXK];
    for (int h = 0; h < K; ++h) perm[h] = h;
    for (int a = 1; a < K; ++a)          // insertion sort by label (stable)
        for (int b = a; b > 0 && lab[perm[b - 1]] > lab[perm[b]]; --b) { int t = perm[b]; perm[b] = perm[b - 1]; perm[b - 1] = t; }
    for (int c = 0; c < K; ++c) seg[c] = (c > 0 && lab[perm[c]] == lab[perm[c - 1]]) ? seg[c - 1] : c;
    // within each segment start from ascending vertex index (next_perm enumerates from there)
    for (int c = 0; c < K; ++c)
        for (int b = c; b > seg[c] && perm[b - 1] > perm[b]; --b) { int t = perm[b]; perm[b] = perm[b - 1]; perm[b - 1] = t; }
    uint32_t bc = 0xffffffffu;
    do {
        const uint32_t code = adj_code(K, adj, perm);
        if (code < bc) {
            bc = code;
            for (int c = 0; c < K; ++c) best[c] = perm[c];
        }
    } while (next_label_perm(K, seg, perm));
    unsigned long long l = 0;
    for (int c = 0; c < K; ++c) l |= (unsigned long long)(lab[best[c]] & 0xff) << (8 * (7 - c));
    uint32_t iv = 0;
    for (int c = 0; c < K; ++c) iv |= (uint32_t)c << (3 * best[c]);
    clab = l;
    cadj = bc;
    inv = iv;
}

// The labeled graph a quick-pattern key denotes, in the key's local vertex order (the order the
// extension kernel's accept step uses for that key's positions).
static __device__ __noinline__ void key_graph(int V, int L, uint64_t key, const uint64_t *pat_lab8, const uint64_t *pat_adj8, int &K,
                          int *labH, uint32_t *adjH) {
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
    split_key(key, pid, pidx, i, jpos, cross);
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

__device__ __forceinline__ void decode_code(int K, unsigned long long clab, uint32_t cadj, int *lab, uint32_t *adj) {
    const int np = K * (K - 1) / 2;
    for (int c = 0; c < K; ++c) { lab[c] = (int)(clab >> (8 * (7 - c))) & 0xff; adj[c] = 0; }
    int q = 0;
    for (int c1 = 0; c1 < K; ++c1)
        for (int c2 = c1 + 1; c2 < K; ++c2, ++q)
            if ((cadj >> (np - 1 - q)) & 1u) { adj[c1] |= 1u << c2; adj[c2] |= 1u << c1; }
}


// Orbit representatives of a canonical pattern: rep[c] = the smallest canonical position that
// an automorphism (a label-preserving order with the same adjacency sequence) maps c to.
static __device__ __noinline__ void orbit_reps(int K, unsigned long long clab, uint32_t cadj, int *rep) {
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

// A canonical code of K <= 7 vertices in 63 bits: label of canonical position c at bits
// 6c..6c+5, the adjacency sequence (as canonicalise returns it) from bit 42.  Bit 63 stays clear,
// so no packed code equals FSM_EMPTY_KEY.
FSM_HD uint64_t pack_code(int K, unsigned long long clab, uint32_t cadj) {
    uint64_t k = 0;
    for (int c = 0; c < K; ++c) k |= ((clab >> (8 * (7 - c))) & 63ull) << (6 * c);
    return k | ((uint64_t)cadj << 42);
}

} // namespace fsm
