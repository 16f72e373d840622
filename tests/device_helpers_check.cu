// Host checks of the index and key helpers the extension kernel shares with the host
// (fsm_device.cuh), against brute force: count_below, centre_pairs (the four-vertex cut of the
// centre pairs), quick-pattern key packing, join-graph symmetry, size-3 pattern indices; and of
// the canonicaliser (fsm_canon.cuh: label-order enumeration and the cell search) and its orbit
// representatives, against the minimum over all K! vertex orders and the automorphisms found
// among them, for K up to 9; and of the one-pass level's compact copies (fsm_canon7.cuh)
// against the general ones.  It also prints the sampling hash of a grid of (seed, x, y) for
// tests/test_device_helpers.py to compare with splitmix64 written from its published
// definition.  Host code only.
#include "fsm_canon7.cuh"
#include <cstdio>
#include <cstdlib>
using namespace fsm;

static int fails = 0;
#define CHECK(c) do { if (!(c)) { ++fails; printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #c); } } while (0)

// ---- canonicaliser against brute force over all K! orders
static uint32_t rng_state = 2463534242u;
static uint32_t xrand() {
    rng_state ^= rng_state << 13; rng_state ^= rng_state >> 17; rng_state ^= rng_state << 5;
    return rng_state;
}

// (label sequence, adjacency sequence) of one order, compared lexicographically
static bool order_less(int K, const int *lab, const uint32_t *adj, const int *pa, const int *pb, int &cmp) {
    for (int c = 0; c < K; ++c)
        if (lab[pa[c]] != lab[pb[c]]) { cmp = lab[pa[c]] < lab[pb[c]] ? -1 : 1; return cmp < 0; }
    const uint64_t a = adj_code(K, adj, pa), b = adj_code(K, adj, pb);
    cmp = a < b ? -1 : (a > b ? 1 : 0);
    return cmp < 0;
}

static void check_canon() {
    int graphs = 0;
    for (int K = 1; K <= FSM_MAXK; ++K) {
        const int reps = K <= 6 ? 400 : (K == 7 ? 200 : (K == 8 ? 60 : 25));
        for (int r = 0; r < reps; ++r) {
            // labels from 1-3 values, a random spanning tree plus random extra edges; some
            // graphs are highly symmetric (all labels equal, complete or empty beyond the tree)
            const int nl = 1 + (int)(xrand() % 3);
            int lab[FSM_MAXK];
            uint32_t adj[FSM_MAXK] = {0};
            for (int h = 0; h < K; ++h) lab[h] = (r % 4 == 0) ? 0 : (int)(xrand() % nl) * 7;
            for (int h = 1; h < K; ++h) {
                const int u = (int)(xrand() % h);
                adj[h] |= 1u << u; adj[u] |= 1u << h;
            }
            const int dens = (int)(xrand() % 5);   // 0: tree; 4: complete
            for (int a = 0; a < K; ++a)
                for (int b = a + 1; b < K; ++b)
                    if ((int)(xrand() % 4) < dens) { adj[a] |= 1u << b; adj[b] |= 1u << a; }
            // brute force: the smallest order over all K! of them, and the automorphisms
            int p[FSM_MAXK], bp[FSM_MAXK];
            for (int h = 0; h < K; ++h) p[h] = bp[h] = h;
            int cmp;
            do {
                if (order_less(K, lab, adj, p, bp, cmp))
                    for (int h = 0; h < K; ++h) bp[h] = p[h];
            } while (next_perm(p, K));
            const uint64_t want = adj_code(K, adj, bp);
            unsigned long long wl = 0;
            for (int c = 0; c < K; ++c) wl |= clab_put(c, lab[bp[c]]);
            // both ways, through canonicalise and the cell search directly
            unsigned long long cl;
            uint64_t ca, inv;
            canonicalise(K, lab, adj, cl, ca, inv);
            CHECK(ca == want && cl == wl);
            int ord[FSM_MAXK], best[FSM_MAXK];
            CHECK(canon_search(K, lab, adj, -1, best) == want);
            for (int c = 0; c < K; ++c) ord[c] = best[c];
            CHECK(adj_code(K, adj, ord) == want);
            for (int c = 0; c < K; ++c) CHECK(lab[best[c]] == clab_get(wl, c));
            // inv maps every vertex to its position in an optimal order
            uint32_t used = 0;
            for (int h = 0; h < K; ++h) {
                const int c = nib_get(inv, h);
                CHECK(c < K && !((used >> c) & 1u));
                used |= 1u << c;
                ord[c] = h;
            }
            CHECK(adj_code(K, adj, ord) == want);
            // an isomorphic copy (vertices renamed) has the same code
            int q[FSM_MAXK], lab2[FSM_MAXK];
            uint32_t adj2[FSM_MAXK] = {0};
            for (int h = 0; h < K; ++h) q[h] = h;
            for (int h = K - 1; h > 0; --h) { const int j = (int)(xrand() % (h + 1)); const int t = q[h]; q[h] = q[j]; q[j] = t; }
            for (int h = 0; h < K; ++h) {
                lab2[q[h]] = lab[h];
                for (int w = 0; w < K; ++w) if ((adj[h] >> w) & 1u) adj2[q[h]] |= 1u << q[w];
            }
            unsigned long long cl2;
            uint64_t ca2, inv2;
            canonicalise(K, lab2, adj2, cl2, ca2, inv2);
            CHECK(ca2 == want && cl2 == wl);
            // orbit representatives against the automorphisms of the canonical graph
            int clb[FSM_MAXK], rep[FSM_MAXK], wrep[FSM_MAXK];
            uint32_t cad[FSM_MAXK];
            decode_code(K, cl, ca, clb, cad);
            for (int c = 0; c < K; ++c) { p[c] = c; wrep[c] = c; }
            do {
                bool aut = true;
                for (int c = 0; c < K && aut; ++c) aut = clb[p[c]] == clb[c];
                if (aut && adj_code(K, cad, p) == ca)
                    for (int c = 0; c < K; ++c) if (p[c] < wrep[c]) wrep[c] = p[c];
            } while (next_perm(p, K));
            orbit_reps(K, cl, ca, rep);
            for (int c = 0; c < K; ++c) CHECK(rep[c] == wrep[c]);
            ++graphs;
        }
    }
    // the search and the marked orbits against label-order enumeration, on many more graphs
    // with two or three labels (few enough label-preserving orders to enumerate)
    for (int K = 4; K <= FSM_MAXK; ++K)
        for (int r = 0; r < 3000; ++r) {
            const int nl = 2 + (int)(xrand() % 2);
            int lab[FSM_MAXK];
            uint32_t adj[FSM_MAXK] = {0};
            for (int h = 0; h < K; ++h) lab[h] = (int)(xrand() % nl);
            for (int h = 1; h < K; ++h) {
                const int u = (int)(xrand() % h);
                adj[h] |= 1u << u; adj[u] |= 1u << h;
            }
            const int dens = (int)(xrand() % 5);
            for (int a = 0; a < K; ++a)
                for (int b = a + 1; b < K; ++b)
                    if ((int)(xrand() % 4) < dens) { adj[a] |= 1u << b; adj[b] |= 1u << a; }
            int perm[FSM_MAXK], seg[FSM_MAXK], best[FSM_MAXK];
            label_sort(K, lab, perm, seg);
            uint64_t bc = ~0ull;
            do { const uint64_t x = adj_code(K, adj, perm); if (x < bc) bc = x; } while (next_label_perm(K, seg, perm));
            CHECK(canon_search(K, lab, adj, -1, best) == bc);
            // orbits of the canonical graph: enumeration and marking
            unsigned long long cl;
            uint64_t ca, inv;
            canonicalise(K, lab, adj, cl, ca, inv);
            int clb[FSM_MAXK], cseg[FSM_MAXK], p[FSM_MAXK], rep[FSM_MAXK], wrep[FSM_MAXK];
            uint32_t cad[FSM_MAXK];
            decode_code(K, cl, ca, clb, cad);
            for (int c = 0; c < K; ++c) {
                p[c] = c; wrep[c] = c;
                cseg[c] = (c > 0 && clb[c] == clb[c - 1]) ? cseg[c - 1] : c;
            }
            do {
                if (adj_code(K, cad, p) == ca)
                    for (int c = 0; c < K; ++c) if (p[c] < wrep[c]) wrep[c] = p[c];
            } while (next_label_perm(K, cseg, p));
            orbit_reps_search(K, clb, cad, cseg, rep);
            for (int c = 0; c < K; ++c) CHECK(rep[c] == wrep[c]);
            ++graphs;
        }
    // the one-pass level's compact routines (K <= 7) give the same codes, orders, orbits and
    // packed codes as the general ones, and decode keys to the same graphs
    for (int K = 1; K <= 7; ++K)
        for (int r = 0; r < 3000; ++r) {
            const int nl = 1 + (int)(xrand() % 3);
            int lab[FSM_MAXK];
            uint32_t adj[FSM_MAXK] = {0};
            for (int h = 0; h < K; ++h) lab[h] = (int)(xrand() % nl) * 21;
            for (int h = 1; h < K; ++h) {
                const int u = (int)(xrand() % h);
                adj[h] |= 1u << u; adj[u] |= 1u << h;
            }
            const int dens = (int)(xrand() % 5);
            for (int a = 0; a < K; ++a)
                for (int b = a + 1; b < K; ++b)
                    if ((int)(xrand() % 4) < dens) { adj[a] |= 1u << b; adj[b] |= 1u << a; }
            unsigned long long cl, cl7;
            uint64_t ca, iv;
            uint32_t ca7, iv7;
            canonicalise(K, lab, adj, cl, ca, iv);
            canonicalise7(K, lab, adj, cl7, ca7, iv7);
            CHECK((uint64_t)ca7 == ca);
            for (int c = 0; c < K; ++c) CHECK((int)((cl7 >> (8 * (7 - c))) & 0xff) == clab_get(cl, c));
            for (int h = 0; h < K; ++h) CHECK((int)((iv7 >> (3 * h)) & 7u) == nib_get(iv, h));
            CHECK(pack_code7(K, cl7, ca7) == pack_code(K, cl, ca));
            int rep[FSM_MAXK], rep7[8];
            orbit_reps(K, cl, ca, rep);
            orbit_reps7(K, cl7, ca7, rep7);
            for (int c = 0; c < K; ++c) CHECK(rep[c] == rep7[c]);
            ++graphs;
        }
    {
        // keys of joins from size-l embeddings (l <= 5) decode to the same graph both ways
        uint64_t plab[16], padj[16];
        for (int P = 0; P < 16; ++P) {
            const int L = 1 + P % 5;
            uint32_t rows[8] = {0};
            for (int h = 1; h < L; ++h) {
                const int u = (int)(xrand() % h);
                rows[h] |= 1u << u; rows[u] |= 1u << h;
            }
            plab[P] = padj[P] = 0;
            for (int h = 0; h < L; ++h) {
                plab[P] |= (uint64_t)(xrand() % 64) << (8 * h);
                padj[P] |= (uint64_t)rows[h] << (8 * h);
            }
        }
        for (int it = 0; it < 20000; ++it) {
            const int P = (int)(xrand() % 16), L = 1 + P % 5;
            const int V = (int)(xrand() % 3);   // two-vertex, single-vertex, edge-list
            const int i = (int)(xrand() % L);
            uint64_t key;
            if (V == FSM_EXPLORE_TV_EDGELIST) {
                key = xrand() & ((1ull << 42) - 1);
                key |= ((uint64_t)xrand() & ((1u << ((L + 2) * (L + 1) / 2)) - 1u)) << 42;
            } else if (V == FSM_EXPLORE_SV) {
                key = make_key((uint32_t)P, xrand() % 64, i, 3, xrand() & ((1u << (L - 1)) - 1u), L);
            } else {
                const int shape = (int)(xrand() % 2), jpos = (int)(xrand() % 3);
                const uint32_t pidx = piece_index(shape, xrand() % 64, xrand() % 64, xrand() % 64);
                key = make_key((uint32_t)P, pidx, i, jpos, xrand() & ((1u << (2 * (L - 1))) - 1u), L);
            }
            int K1, K2, l1[FSM_MAXK], l2[8];
            uint32_t a1[FSM_MAXK], a2[8];
            key_graph(V, L, key, plab, padj, K1, l1, a1);
            key_graph7(V, L, key, plab, padj, K2, l2, a2);
            CHECK(K1 == K2);
            for (int h = 0; h < K1 && h < 8; ++h) CHECK(l1[h] == l2[h] && a1[h] == a2[h]);
        }
    }
    // highly symmetric unlabeled 9-vertex graphs (the cell search's hardest cases): K_9, C_9,
    // the 3x3 rook graph, K_{3,3,3}, the Petersen graph minus a vertex, the 3-cube plus a hub;
    // each against the brute-force minimum, with its orbits
    {
        const int K = 9;
        uint32_t g[6][9] = {};
        for (int a = 0; a < K; ++a)
            for (int b = 0; b < K; ++b) {
                if (a == b) continue;
                g[0][a] |= 1u << b;                                                  // K_9
                if ((a + 1) % K == b || (b + 1) % K == a) g[1][a] |= 1u << b;        // C_9
                if (a / 3 == b / 3 || a % 3 == b % 3) g[2][a] |= 1u << b;            // rook 3x3
                if (a / 3 != b / 3) g[3][a] |= 1u << b;                              // K_{3,3,3}
            }
        // Petersen graph (outer 5-cycle 0..4, spokes i - i+5, inner pentagram) minus vertex 9
        const int pe[15][2] = {{0,1},{1,2},{2,3},{3,4},{4,0},{0,5},{1,6},{2,7},{3,8},{4,9},{5,7},{7,9},{9,6},{6,8},{8,5}};
        for (auto &e : pe)
            if (e[0] < 9 && e[1] < 9) { g[4][e[0]] |= 1u << e[1]; g[4][e[1]] |= 1u << e[0]; }
        // 3-cube on 0..7 plus vertex 8 joined to all of it
        for (int a = 0; a < 8; ++a) {
            for (int bit = 0; bit < 3; ++bit) g[5][a] |= 1u << (a ^ (1 << bit));
            g[5][a] |= 1u << 8;
            g[5][8] |= 1u << a;
        }
        int lab[9] = {0};
        for (int q = 0; q < 6; ++q) {
            int p[9];
            for (int h = 0; h < K; ++h) p[h] = h;
            uint64_t want = adj_code(K, g[q], p);
            do {
                const uint64_t x = adj_code(K, g[q], p);
                if (x < want) want = x;
            } while (next_perm(p, K));
            unsigned long long cl;
            uint64_t ca, inv;
            canonicalise(K, lab, g[q], cl, ca, inv);
            CHECK(ca == want);
            int clb[9], rep[9], wrep[9];
            uint32_t cad[9];
            decode_code(K, cl, ca, clb, cad);
            for (int c = 0; c < K; ++c) { p[c] = c; wrep[c] = c; }
            do {
                if (adj_code(K, cad, p) == ca)
                    for (int c = 0; c < K; ++c) if (p[c] < wrep[c]) wrep[c] = p[c];
            } while (next_perm(p, K));
            orbit_reps(K, cl, ca, rep);
            for (int c = 0; c < K; ++c) CHECK(rep[c] == wrep[c]);
            ++graphs;
        }
    }
    printf("canonical codes checked on %d graphs\n", graphs);
}

int main() {
    // count_below on sorted lists with gaps
    for (int n = 0; n <= 40; ++n) {
        int32_t a[40];
        for (int q = 0; q < n; ++q) a[q] = 3 * q + (q % 2);
        for (int x = -2; x <= 3 * n + 3; ++x) {
            int brute = 0;
            for (int q = 0; q < n; ++q) brute += a[q] < x;
            CHECK(count_below(a, n, x) == brute);
        }
    }
    // centre_pairs(d, c) = #{(x, y): 0 <= x < y < d, x < c}
    for (int d = 0; d <= 60; ++d)
        for (int c = 0; c <= d; ++c) {
            long brute = 0;
            for (int y = 0; y < d; ++y)
                for (int x = 0; x < y; ++x) brute += x < c;
            CHECK(centre_pairs(d, c) == brute);
        }
    // quick-pattern keys: fields round-trip at every level size (10 cross bits up to l = 6, 12
    // at l = 7), the narrow layout is the one of 10-bit cross fields, and the packed key never
    // equals the empty key
    unsigned s = 12345u;
    for (int it = 0; it < 100000; ++it) {
        const int L = 1 + it % 7;
        s = s * 1103515245u + 12345u; const uint32_t pid = (s >> 4) & ((1u << 24) - 1);
        s = s * 1103515245u + 12345u; const uint32_t pidx = (s >> 3) & ((1u << 19) - 1);
        s = s * 1103515245u + 12345u; const int i = (int)((s >> 5) % 7), j = (int)((s >> 9) % 4);
        s = s * 1103515245u + 12345u; const uint32_t cross = (s >> 7) & ((1u << (L >= 7 ? 12 : 10)) - 1u);
        const uint64_t key = make_key(pid, pidx, i, j, cross, L);
        uint32_t p2, x2, c2; int i2, j2;
        split_key(key, L, p2, x2, i2, j2, c2);
        CHECK(p2 == pid && x2 == pidx && i2 == i && j2 == j && c2 == cross);
        CHECK(key != FSM_EMPTY_KEY);
        if (L <= 6)
            CHECK(key == (((uint64_t)pid << 34) | ((uint64_t)pidx << 15) | ((uint64_t)i << 12) | ((uint64_t)j << 10) | cross));
    }
    // join graphs are symmetric and loop-free for every level size, shape, join position,
    // key position and cross subset (s = a path over its l positions)
    for (int L = 2; L <= 7; ++L)
        for (int shape = 0; shape < 2; ++shape)
            for (int jpos = 0; jpos < 3; ++jpos)
                for (int i = 0; i < L; ++i)
                    for (uint32_t sub = 0; sub < (1u << (2 * (L - 1))); ++sub) {
                        uint64_t srows = 0;
                        for (int h = 0; h + 1 < L; ++h) {
                            srows |= (uint64_t)(1u << (h + 1)) << (8 * h);
                            srows |= (uint64_t)(1u << h) << (8 * (h + 1));
                        }
                        uint32_t tj0, tj1, txx, adj[FSM_MAXK];
                        piece_join_edges(shape, jpos, tj0, tj1, txx);
                        join_graph(L, srows, i, tj0, tj1, txx, sub, adj);
                        const int K = L + 2;
                        for (int u = 0; u < K; ++u) {
                            CHECK(!(adj[u] >> u & 1u));
                            for (int w = 0; w < K; ++w) CHECK(((adj[u] >> w) & 1u) == ((adj[w] >> u) & 1u));
                        }
                        CHECK(mask_connected((1u << K) - 1u, adj, K));
                    }
    // size-3 pattern indices: a wedge's ends are unordered, a triangle's vertices too
    for (int a = 0; a < 64; a += 7)
        for (int b = 0; b < 64; b += 5)
            for (int c = 0; c < 64; c += 3) {
                CHECK(wedge_index(a, b, c) == wedge_index(a, c, b));
                const uint32_t t = tri_index(a, b, c);
                CHECK(t == tri_index(a, c, b) && t == tri_index(b, a, c) && t == tri_index(b, c, a) &&
                      t == tri_index(c, a, b) && t == tri_index(c, b, a));
                CHECK(t != wedge_index(a, b, c));
            }
    // pattern words round-trip
    for (int c = 0; c < FSM_MAXK; ++c)
        for (int l = 0; l < 64; ++l) {
            CHECK(clab_get(clab_put(c, l), c) == l);
            for (int c2 = 0; c2 < FSM_MAXK; ++c2)
                if (c2 != c) CHECK(clab_get(clab_put(c, l), c2) == 0);
        }
    for (int h = 0; h < FSM_MAXK; ++h)
        for (int v = 0; v < 16; ++v) CHECK(nib_get(nib_put(h, v) | nib_put((h + 1) % FSM_MAXK, 15 - v), h) == v);
    check_canon();
    // sampling hash of a grid, for the splitmix64 comparison
    const uint64_t seeds[3] = {0ull, 1ull, 0x123456789abcdefull};
    const int32_t xs[4] = {0, 1, 77, 2147483647};
    for (uint64_t sd : seeds)
        for (int32_t x : xs)
            for (int32_t y : xs) {
                uint64_t h = splitmix_step(sd);
                h = splitmix_step(h ^ (uint64_t)(uint32_t)x);
                h = splitmix_step(h ^ (uint64_t)(uint32_t)y);
                CHECK(keep_edge(sd, h + 1, x, y) && !keep_edge(sd, h, x, y));
                printf("hash %llu %d %d %llu\n", (unsigned long long)sd, x, y, (unsigned long long)h);
            }
    printf("fails %d\n", fails);
    return fails != 0;
}
