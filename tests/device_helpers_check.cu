// Host checks of the index and key helpers the extension kernel shares with the host
// (fsm_device.cuh), against brute force: count_below, centre_pairs (the four-vertex cut of the
// centre pairs), quick-pattern key packing, join-graph symmetry, size-3 pattern indices.  It
// also prints the sampling hash of a grid of (seed, x, y) for tests/test_device_helpers.py to
// compare with splitmix64 written from its published definition.  Host code only.
#include "fsm_device.cuh"
#include <cstdio>
#include <cstdlib>
using namespace fsm;

static int fails = 0;
#define CHECK(c) do { if (!(c)) { ++fails; printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #c); } } while (0)

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
    // quick-pattern keys: fields round-trip and the packed key never equals the empty key
    unsigned s = 12345u;
    for (int it = 0; it < 100000; ++it) {
        s = s * 1103515245u + 12345u; const uint32_t pid = (s >> 4) & ((1u << 24) - 1);
        s = s * 1103515245u + 12345u; const uint32_t pidx = (s >> 3) & ((1u << 19) - 1);
        s = s * 1103515245u + 12345u; const int i = (int)((s >> 5) % 7), j = (int)((s >> 9) % 3);
        s = s * 1103515245u + 12345u; const uint32_t cross = (s >> 7) & 1023u;
        const uint64_t key = make_key(pid, pidx, i, j, cross);
        uint32_t p2, x2, c2; int i2, j2;
        split_key(key, p2, x2, i2, j2, c2);
        CHECK(p2 == pid && x2 == pidx && i2 == i && j2 == j && c2 == cross);
        CHECK(key != FSM_EMPTY_KEY);
    }
    // join graphs are symmetric and loop-free for every level size, shape, join position,
    // key position and cross subset (s = a path over its l positions)
    for (int L = 2; L <= 6; ++L)
        for (int shape = 0; shape < 2; ++shape)
            for (int jpos = 0; jpos < 3; ++jpos)
                for (int i = 0; i < L; ++i)
                    for (uint32_t sub = 0; sub < (1u << (2 * (L - 1))); ++sub) {
                        uint64_t srows = 0;
                        for (int h = 0; h + 1 < L; ++h) {
                            srows |= (uint64_t)(1u << (h + 1)) << (8 * h);
                            srows |= (uint64_t)(1u << h) << (8 * (h + 1));
                        }
                        uint32_t tj0, tj1, txx, adj[8];
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
