// Host check of the four-vertex dissection closed form (dissect4_keeps) against the general
// smallest-vertex-first dissection (dissect3, Algorithm 1): every key position, piece shape,
// join position, cross-edge subset and order of the four vertex ids.  Built and run by
// tests/test_dissect4.py; host code only.
#include "fsm_extend.cuh"
#include <cstdio>
using namespace fsm;
int main() {
    long checked = 0, bad = 0, kept = 0;
    // all id orders: permutations of 4 ids
    int ids[24][4]; int np = 0;
    for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) for (int c = 0; c < 4; ++c) for (int d = 0; d < 4; ++d)
        if (a != b && a != c && a != d && b != c && b != d && c != d) { ids[np][0]=a; ids[np][1]=b; ids[np][2]=c; ids[np][3]=d; ++np; }
    for (int i = 0; i < 2; ++i)
    for (int shape = 0; shape < 2; ++shape)
    for (int jpos = 0; jpos < 3; ++jpos)
    for (uint32_t sub = 0; sub < 4; ++sub)
    for (int q = 0; q < np; ++q) {
        uint32_t tj0, tj1, txx;
        piece_join_edges(shape, jpos, tj0, tj1, txx);
        uint64_t srows = (uint64_t)0x2 | ((uint64_t)0x1 << 8);   // s = edge {0, 1}
        uint32_t adjK[4];
        join_graph(2, srows, i, tj0, tj1, txx, sub, adjK);
        int32_t gid[4] = {ids[q][0], ids[q][1], ids[q][2], ids[q][3]};
        uint32_t lm = 0; int jn = -1;
        dissect3(4, gid, adjK, lm, jn);
        const bool ref = (lm == ((1u << i) | 12u)) && jn == i;
        const bool got = dissect4_keeps(gid, adjK, i);
        ++checked; kept += ref; if (ref != got) ++bad;
    }
    printf("checked %ld kept %ld mismatches %ld\n", checked, kept, bad);
    return bad != 0;
}
