// fsm_canon7.cuh -- canonical codes for the one-pass last level (K <= 7 vertices).
//
// The same canonical form as fsm_canon.cuh (the smallest (label sequence, adjacency sequence)
// over all vertex orders, found by enumerating the label-preserving orders of the label-sorted
// positions), in the compact words this level has always used: label bytes (byte 7 - c holds
// canonical position c), a 32-bit adjacency word (at most 21 pair bits, first pair most
// significant) and 3-bit vertex orders, with 8-entry scratch arrays.  The one-pass kernel calls
// only these on first sight of a quick pattern, so its code stays what it was before patterns of
// 8 and 9 vertices needed the wider words and the cell search of fsm_canon.cuh.  The host build
// of tests/device_helpers_check.cu checks them against fsm_canon.cuh.
#pragma once
#include "fsm_canon.cuh"

namespace fsm {

FSM_HD uint32_t adj_code7(int K, const uint32_t *adj, const int *perm) {
    uint32_t code = 0;
    for (int c1 = 0; c1 < K; ++c1) {
        const uint32_t row = adj[perm[c1]];
        for (int c2 = c1 + 1; c2 < K; ++c2) code = (code << 1) | ((row >> perm[c2]) & 1u);
    }
    return code;
}

// clab7: label of canonical position c in byte 7 - c; cadj7: adjacency word; inv7: vertex h ->
// canonical position in bits 3h..3h+2 (first optimal order).
static __host__ __device__ __noinline__ void canonicalise7(int K, const int *lab, const uint32_t *adj,
                                                           unsigned long long &clab7, uint32_t &cadj7, uint32_t &inv7) {
    int perm[8], seg[8], best[8];
    for (int h = 0; h < K; ++h) perm[h] = h;
    for (int a = 1; a < K; ++a)          // insertion sort by label (stable)
        for (int b = a; b > 0 && lab[perm[b - 1]] > lab[perm[b]]; --b) { int t = perm[b]; perm[b] = perm[b - 1]; perm[b - 1] = t; }
    for (int c = 0; c < K; ++c) seg[c] = (c > 0 && lab[perm[c]] == lab[perm[c - 1]]) ? seg[c - 1] : c;
    // within each segment start from ascending vertex index (next_perm enumerates from there)
    for (int c = 0; c < K; ++c)
        for (int b = c; b > seg[c] && perm[b - 1] > perm[b]; --b) { int t = perm[b]; perm[b] = perm[b - 1]; perm[b - 1] = t; }
    uint32_t bc = 0xffffffffu;
    do {
        const uint32_t code = adj_code7(K, adj, perm);
        if (code < bc) {
            bc = code;
            for (int c = 0; c < K; ++c) best[c] = perm[c];
        }
    } while (next_label_perm(K, seg, perm));
    unsigned long long l = 0;
    for (int c = 0; c < K; ++c) l |= (unsigned long long)(lab[best[c]] & 0xff) << (8 * (7 - c));
    uint32_t iv = 0;
    for (int c = 0; c < K; ++c) iv |= (uint32_t)c << (3 * best[c]);
    clab7 = l;
    cadj7 = bc;
    inv7 = iv;
}

// The labeled graph of a key of a join from a size-l embedding, l <= 5 (the narrow key layout),
// in the key's local vertex order; as key_graph of fsm_canon.cuh.
static __host__ __device__ __noinline__ void key_graph7(int V, int L, uint64_t key, const uint64_t *pat_lab8,
                                                        const uint64_t *pat_adj8, int &K, int *labH, uint32_t *adjH) {
    if (V == FSM_EXPLORE_TV_EDGELIST) {
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
    split_key(key, 1, pid, pidx, i, jpos, cross);   // any level size below 7: the narrow layout
    const uint64_t lab8 = pat_lab8[pid], srows = pat_adj8[pid];
    for (int h = 0; h < L; ++h) labH[h] = (int)(lab8 >> (8 * h)) & 0xff;
    if (V == FSM_EXPLORE_SV) {
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

FSM_HD void decode_code7(int K, unsigned long long clab7, uint32_t cadj7, int *lab, uint32_t *adj) {
    const int np = K * (K - 1) / 2;
    for (int c = 0; c < K; ++c) { lab[c] = (int)(clab7 >> (8 * (7 - c))) & 0xff; adj[c] = 0; }
    int q = 0;
    for (int c1 = 0; c1 < K; ++c1)
        for (int c2 = c1 + 1; c2 < K; ++c2, ++q)
            if ((cadj7 >> (np - 1 - q)) & 1u) { adj[c1] |= 1u << c2; adj[c2] |= 1u << c1; }
}

// Orbit representatives (as orbit_reps of fsm_canon.cuh), by enumeration.
static __host__ __device__ __noinline__ void orbit_reps7(int K, unsigned long long clab7, uint32_t cadj7, int *rep) {
    int lab[8], perm[8], seg[8];
    uint32_t adj[8];
    decode_code7(K, clab7, cadj7, lab, adj);
    for (int c = 0; c < K; ++c) {
        perm[c] = c;
        rep[c] = c;
        seg[c] = (c > 0 && lab[c] == lab[c - 1]) ? seg[c - 1] : c;
    }
    do {
        if (adj_code7(K, adj, perm) == cadj7)
            for (int c = 0; c < K; ++c) if (perm[c] < rep[c]) rep[c] = perm[c];
    } while (next_label_perm(K, seg, perm));
}

// pack_code of fsm_canon.cuh from the compact words: the same 63-bit value.
FSM_HD uint64_t pack_code7(int K, unsigned long long clab7, uint32_t cadj7) {
    uint64_t k = 0;
    for (int c = 0; c < K; ++c) k |= ((clab7 >> (8 * (7 - c))) & 63ull) << (6 * c);
    return k | ((uint64_t)cadj7 << 42);
}

} // namespace fsm
