/*
 * Plain CPU oracle for exact frequent subgraph mining (FSM) under MNI support.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load this file.  It shares no code with the CUDA library: it computes the
 * problem from its definitions, slowly and directly.
 *
 * What it computes (paper Section 2):
 *   - Section 2.1: a subgraph G'=(V',E') of G has V' in V, E' in E and inherits labels;
 *     vertex-induced means E' holds every edge of G among V'; edge-induced embeddings are the
 *     connected (V',E') with E' any subset of the induced edges (reading of the garbled
 *     definition: every connected edge subset, the full one included).
 *   - Definition 1 (isomorphism), read as label-preserving: two labeled graphs share a pattern
 *     when a bijection preserves both adjacency and vertex labels.
 *   - Definition 2 (MNI support): sigma(P) = min over pattern vertices c of the number of
 *     distinct images f(c), f ranging over every isomorphism from P onto an embedding of P.
 *   - Section 2.2 problem statement: report every pattern with |V_P| = k and sigma >= t.
 *
 * Method, step by step (no step of the paper's own exploration is used here):
 *   1. Every connected k-vertex set of G is listed exactly once with the ESU algorithm
 *      (Wernicke, "Efficient detection of network motifs", 2006): each set is grown from its
 *      smallest vertex v, the extension set holding only vertices > v that are exclusive
 *      neighbours of the newest vertex.
 *   2. For a set u_0 < ... < u_{k-1}, the embeddings are (V', E') with E' = all induced edges
 *      (vertex-induced) or every connected spanning subset of them (edge-induced).
 *   3. Canonical code: for a permutation pi of the k positions, code(pi) is the sequence
 *      (L(u_pi0), ..., L(u_pi(k-1)), A(pi0,pi1), A(pi0,pi2), ..., A(pi(k-2),pi(k-1))) with A
 *      the 0/1 adjacency of the embedding and pairs (c1 < c2) in row-major order.  The
 *      canonical code of the embedding is the lexicographic minimum over all k! permutations.
 *      Equal codes <=> isomorphic (label-preserving) graphs.
 *   4. Every permutation attaining the minimum is an isomorphism from the canonical pattern
 *      onto the embedding (c -> u_pi(c)); for all of them and every canonical position c,
 *      u_pi(c) joins the image set D[P][c].
 *   5. sigma(P) = min_c |D[P][c]|; patterns with sigma >= t are returned sorted by code.
 *
 * Results are memoised per raw (label tuple, adjacency) key so the k! scan runs once per
 * distinct raw key.  Image sets are growable open-addressing hash sets of vertex ids.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXK 9

/* ------------------------------------------------------------------ small utilities */

static int adjacent(const int32_t *row_ptr, const int32_t *col, int32_t a, int32_t b) {
    int32_t lo = row_ptr[a], hi = row_ptr[a + 1] - 1;
    while (lo <= hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (col[mid] == b) return 1;
        if (col[mid] < b) lo = mid + 1; else hi = mid - 1;
    }
    return 0;
}

static uint64_t mix64(uint64_t x) {
    x ^= x >> 33; x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33; return x;
}

/* growable hash set of int32 vertex ids (value -1 marks an empty slot) */
typedef struct { int32_t *slot; int64_t cap, size; } vset_t;

static void vset_init(vset_t *s) { s->slot = NULL; s->cap = 0; s->size = 0; }

static void vset_insert(vset_t *s, int32_t x);

static void vset_grow(vset_t *s) {
    int64_t ncap = s->cap ? s->cap * 2 : 16;
    int32_t *old = s->slot; int64_t ocap = s->cap;
    s->slot = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncap);
    for (int64_t i = 0; i < ncap; i++) s->slot[i] = -1;
    s->cap = ncap; s->size = 0;
    for (int64_t i = 0; i < ocap; i++) if (old[i] >= 0) vset_insert(s, old[i]);
    free(old);
}

static void vset_insert(vset_t *s, int32_t x) {
    if ((s->size + 1) * 2 > s->cap) vset_grow(s);
    uint64_t h = mix64((uint64_t)(uint32_t)x) & (uint64_t)(s->cap - 1);
    while (s->slot[h] >= 0) {
        if (s->slot[h] == x) return;
        h = (h + 1) & (uint64_t)(s->cap - 1);
    }
    s->slot[h] = x; s->size++;
}

/* ------------------------------------------------------------------ canonical codes */

/* A code is the label sequence plus the adjacency sequence packed into an integer whose most
 * significant used bit is the first pair (0,1); integer order equals sequence order. */
typedef struct { int32_t lab[OR_MAXK]; uint64_t adj; } code_t;

static int code_cmp(const code_t *a, const code_t *b, int k) {
    for (int i = 0; i < k; i++)
        if (a->lab[i] != b->lab[i]) return a->lab[i] < b->lab[i] ? -1 : 1;
    if (a->adj != b->adj) return a->adj < b->adj ? -1 : 1;
    return 0;
}

typedef struct {
    int k, npairs, nperm;
    uint8_t *perms;                 /* nperm x k, all permutations of 0..k-1 */
    int pi[OR_MAXK * OR_MAXK];      /* pair index of (c1, c2), c1 < c2 */
} canon_ctx_t;

static void gen_perms(canon_ctx_t *cx) {
    int k = cx->k, f = 1;
    for (int i = 2; i <= k; i++) f *= i;
    cx->nperm = f;
    cx->perms = (uint8_t *)malloc((size_t)f * (size_t)(k ? k : 1));
    uint8_t a[OR_MAXK];
    for (int i = 0; i < k; i++) a[i] = (uint8_t)i;
    for (int p = 0; p < f; p++) {
        memcpy(cx->perms + (size_t)p * k, a, (size_t)k);
        /* next lexicographic permutation */
        int i = k - 2;
        while (i >= 0 && a[i] > a[i + 1]) i--;
        if (i < 0) break;
        int j = k - 1;
        while (a[j] < a[i]) j--;
        uint8_t t = a[i]; a[i] = a[j]; a[j] = t;
        for (int l = i + 1, r = k - 1; l < r; l++, r--) { t = a[l]; a[l] = a[r]; a[r] = t; }
    }
    int q = 0;
    for (int c1 = 0; c1 < k; c1++)
        for (int c2 = c1 + 1; c2 < k; c2++) cx->pi[c1 * OR_MAXK + c2] = q++;
    cx->npairs = q;
}

/* code of permutation perm applied to (lab, adjrow): position c holds vertex perm[c] */
static void code_of(const canon_ctx_t *cx, const uint8_t *perm, const int32_t *lab,
                    const uint32_t *adjrow, code_t *out) {
    int k = cx->k;
    for (int c = 0; c < k; c++) out->lab[c] = lab[perm[c]];
    for (int c = k; c < OR_MAXK; c++) out->lab[c] = 0;
    uint64_t a = 0;
    for (int c1 = 0; c1 < k; c1++)
        for (int c2 = c1 + 1; c2 < k; c2++)
            a = (a << 1) | (uint64_t)((adjrow[perm[c1]] >> perm[c2]) & 1u);
    out->adj = a;
}

/* code_cmp(code of perm, *c): the label sequence first, then the adjacency sequence, from
 * the first position and pair on, returning at the first difference */
static int perm_cmp(const canon_ctx_t *cx, const uint8_t *perm, const int32_t *lab, const uint32_t *adjrow,
                    const code_t *c) {
    int k = cx->k;
    for (int i = 0; i < k; i++)
        if (lab[perm[i]] != c->lab[i]) return lab[perm[i]] < c->lab[i] ? -1 : 1;
    int q = cx->npairs - 1;
    for (int c1 = 0; c1 < k; c1++)
        for (int c2 = c1 + 1; c2 < k; c2++, q--) {
            const uint64_t a = (adjrow[perm[c1]] >> perm[c2]) & 1u, b = (c->adj >> q) & 1u;
            if (a != b) return a < b ? -1 : 1;
        }
    return 0;
}

/* ------------------------------------------------------------------ pattern registry */

typedef struct {
    code_t code;
    int64_t count;                  /* embeddings (V', E') of this pattern */
    vset_t dom[OR_MAXK];            /* D[P][c] */
    int64_t scount;                 /* sampled mode: kept embeddings */
    vset_t sdom[OR_MAXK];           /* sampled mode: images over kept embeddings */
} pattern_t;

typedef struct {
    uint64_t key_lab, key_lab2, key_adj; int used;   /* raw key: labels 0..7, labels 8.., pairs */
    int32_t pattern;                /* index into patterns */
    int32_t nopt; int64_t perm_off; /* optimal permutations, k bytes each, in perm pool */
} memo_t;

typedef struct {
    int k, mode;
    const int32_t *row_ptr, *col, *labels;
    int32_t n;
    int64_t budget, seen;           /* stop after `budget` embeddings (<= 0: no limit) */
    int stop;
    /* sampled mode: an embedding is kept iff the 3-vertex part of its dissection is kept */
    int sampled;
    uint64_t seed, thr;
    canon_ctx_t cx;
    pattern_t *pat; int64_t npat, cappat;
    /* pattern lookup by canonical code: open addressing over indices */
    int32_t *pat_slot; int64_t pat_cap;
    memo_t *memo; int64_t memo_cap, memo_size;
    uint8_t *pool; int64_t pool_size, pool_cap;
} oracle_t;

static uint64_t code_hash(const code_t *c, int k) {
    uint64_t h = 0x9e3779b97f4a7c15ULL;
    for (int i = 0; i < k; i++) h = mix64(h ^ (uint64_t)(uint32_t)c->lab[i]);
    return mix64(h ^ c->adj);
}

static int32_t pattern_find_or_add(oracle_t *o, const code_t *c) {
    if ((o->npat + 1) * 2 > o->pat_cap) {
        int64_t ncap = o->pat_cap ? o->pat_cap * 2 : 64;
        free(o->pat_slot);
        o->pat_slot = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncap);
        for (int64_t i = 0; i < ncap; i++) o->pat_slot[i] = -1;
        o->pat_cap = ncap;
        for (int64_t p = 0; p < o->npat; p++) {
            uint64_t h = code_hash(&o->pat[p].code, o->k) & (uint64_t)(ncap - 1);
            while (o->pat_slot[h] >= 0) h = (h + 1) & (uint64_t)(ncap - 1);
            o->pat_slot[h] = (int32_t)p;
        }
    }
    uint64_t h = code_hash(c, o->k) & (uint64_t)(o->pat_cap - 1);
    while (o->pat_slot[h] >= 0) {
        if (code_cmp(&o->pat[o->pat_slot[h]].code, c, o->k) == 0) return o->pat_slot[h];
        h = (h + 1) & (uint64_t)(o->pat_cap - 1);
    }
    if (o->npat == o->cappat) {
        o->cappat = o->cappat ? o->cappat * 2 : 64;
        o->pat = (pattern_t *)realloc(o->pat, sizeof(pattern_t) * (size_t)o->cappat);
    }
    pattern_t *p = &o->pat[o->npat];
    p->code = *c; p->count = 0; p->scount = 0;
    for (int i = 0; i < OR_MAXK; i++) { vset_init(&p->dom[i]); vset_init(&p->sdom[i]); }
    o->pat_slot[h] = (int32_t)o->npat;
    return (int32_t)o->npat++;
}

static uint64_t memo_hash(uint64_t klab, uint64_t klab2, uint64_t kadj) {
    return mix64(klab ^ mix64(kadj ^ mix64(klab2)));
}

static memo_t *memo_lookup(oracle_t *o, uint64_t klab, uint64_t klab2, uint64_t kadj) {
    if ((o->memo_size + 1) * 2 > o->memo_cap) {
        int64_t ncap = o->memo_cap ? o->memo_cap * 2 : 1024;
        memo_t *old = o->memo; int64_t ocap = o->memo_cap;
        o->memo = (memo_t *)calloc((size_t)ncap, sizeof(memo_t));
        o->memo_cap = ncap;
        for (int64_t i = 0; i < ocap; i++) if (old[i].used) {
            uint64_t h = memo_hash(old[i].key_lab, old[i].key_lab2, old[i].key_adj) & (uint64_t)(ncap - 1);
            while (o->memo[h].used) h = (h + 1) & (uint64_t)(ncap - 1);
            o->memo[h] = old[i];
        }
        free(old);
    }
    uint64_t h = memo_hash(klab, klab2, kadj) & (uint64_t)(o->memo_cap - 1);
    while (o->memo[h].used) {
        if (o->memo[h].key_lab == klab && o->memo[h].key_lab2 == klab2 && o->memo[h].key_adj == kadj)
            return &o->memo[h];
        h = (h + 1) & (uint64_t)(o->memo_cap - 1);
    }
    memo_t *m = &o->memo[h];
    m->used = 1; m->key_lab = klab; m->key_lab2 = klab2; m->key_adj = kadj; m->pattern = -1;
    o->memo_size++;
    return m;
}

/* canonicalise one raw labeled graph (lab, adjrow over positions 0..k-1), memoised */
static memo_t *canonical(oracle_t *o, const int32_t *lab, const uint32_t *adjrow) {
    int k = o->k;
    uint64_t klab = 0, klab2 = 0, kadj = 0;
    for (int i = 0; i < k; i++) {
        if (i < 8) klab = (klab << 8) | (uint64_t)(lab[i] & 0xff);
        else klab2 = (klab2 << 8) | (uint64_t)(lab[i] & 0xff);
    }
    /* raw key: the label tuple and the packed upper triangle of the adjacency */
    for (int c1 = 0; c1 < k; c1++)
        for (int c2 = c1 + 1; c2 < k; c2++)
            kadj = (kadj << 1) | (uint64_t)((adjrow[c1] >> c2) & 1u);
    memo_t *m = memo_lookup(o, klab, klab2, kadj);
    if (m->pattern >= 0) return m;
    /* the minimum code over all k! permutations, then every permutation attaining it; each
     * comparison is lexicographic and stops at the first differing label or pair */
    code_t best;
    code_of(&o->cx, o->cx.perms, lab, adjrow, &best);
    for (int p = 1; p < o->cx.nperm; p++) {
        const uint8_t *perm = o->cx.perms + (size_t)p * k;
        if (perm_cmp(&o->cx, perm, lab, adjrow, &best) < 0) code_of(&o->cx, perm, lab, adjrow, &best);
    }
    m->perm_off = o->pool_size; m->nopt = 0;
    for (int p = 0; p < o->cx.nperm; p++) {
        const uint8_t *perm = o->cx.perms + (size_t)p * k;
        if (perm_cmp(&o->cx, perm, lab, adjrow, &best) != 0) continue;
        if (o->pool_size + k > o->pool_cap) {
            o->pool_cap = o->pool_cap ? o->pool_cap * 2 : 4096;
            o->pool = (uint8_t *)realloc(o->pool, (size_t)o->pool_cap);
        }
        memcpy(o->pool + o->pool_size, perm, (size_t)k);
        o->pool_size += k;
        m->nopt++;
    }
    m->pattern = pattern_find_or_add(o, &best);
    return m;
}

/* ------------------------------------------------------------------ embeddings of one set */

static int spans_connected(int k, const uint32_t *adjrow) {
    uint32_t seen = 1u, frontier = 1u;
    while (frontier) {
        uint32_t nxt = 0;
        for (int i = 0; i < k; i++) if (frontier >> i & 1u) nxt |= adjrow[i];
        nxt &= ~seen;
        seen |= nxt; frontier = nxt;
    }
    return seen == ((1u << k) - 1u);
}

/* ---- sampled mode: Algorithm 1's dissect (n = 3) and the piece-sampling rule ----
 * dissect: for each start vertex in ascending id order, visit 3 vertices by always adding the
 * smallest id adjacent to the visited ones; the 3-set l is kept if the other vertices plus one
 * vertex v' of l (tried in ascending id order) are connected.  If no start vertex works, take
 * the smallest (sorted ids of l, id of v') over all connected 3-sets l with a connected rest.
 * Positions here are already in ascending id order (u[0] < u[1] < ...). */
static int conn_mask(int k, const uint32_t *adjrow, uint32_t m) {
    if (!m) return 0;
    uint32_t seen = m & (~m + 1u), fr = seen;
    while (fr) {
        uint32_t nx = 0;
        for (int i = 0; i < k; i++) if ((fr >> i) & 1u) nx |= adjrow[i];
        nx &= m & ~seen; seen |= nx; fr = nx;
    }
    return seen == m;
}

static uint32_t dissect_three_join(int k, const uint32_t *adjrow, int *join) {
    uint32_t all = (1u << k) - 1u;
    for (int start = 0; start < k; start++) {
        uint32_t vis = 1u << start;
        for (int step = 0; step < 2; step++) {
            uint32_t cand = 0;
            for (int i = 0; i < k; i++) if ((vis >> i) & 1u) cand |= adjrow[i];
            cand &= all & ~vis;
            if (!cand) { vis = 0; break; }
            vis |= cand & (~cand + 1u);          /* smallest id = lowest position */
        }
        if (!vis) continue;
        for (int v = 0; v < k; v++)
            if (((vis >> v) & 1u) && conn_mask(k, adjrow, (all & ~vis) | (1u << v))) { *join = v; return vis; }
    }
    /* exhaustive rule: smallest sorted triple (a < b < c), then smallest join */
    for (int a = 0; a < k; a++)
        for (int b = a + 1; b < k; b++)
            for (int c = b + 1; c < k; c++) {
                uint32_t l = (1u << a) | (1u << b) | (1u << c);
                if (!conn_mask(k, adjrow, l)) continue;
                int js[3] = {a, b, c};
                for (int q = 0; q < 3; q++)
                    if (conn_mask(k, adjrow, (all & ~l) | (1u << js[q]))) { *join = js[q]; return l; }
            }
    *join = -1;
    return 0;
}

static uint32_t dissect_three(int k, const uint32_t *adjrow) {
    int j;
    return dissect_three_join(k, adjrow, &j);
}

/* splitmix64 (Steele, Lea, Flood 2014): add the golden gamma, then mix */
static uint64_t smix(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* directed edge x -> y kept at rate q: H(H(H(seed) ^ x) ^ y) < floor(q * 2^64) */
static int edge_kept(const oracle_t *o, int32_t x, int32_t y) {
    uint64_t h = smix(o->seed);
    h = smix(h ^ (uint64_t)(uint32_t)x);
    h = smix(h ^ (uint64_t)(uint32_t)y);
    return h < o->thr;
}

/* The 3-vertex part l of the embedding's dissection, seen from its join vertex j: if j is
 * adjacent (in the embedding) to both other vertices x, y of l, the part is kept iff j -> x and
 * j -> y are kept edges; otherwise j is the end of a wedge with centre c and other end z, and
 * the part is kept iff j -> c and c -> z are kept. */
static int kept(const oracle_t *o, const int32_t *u, const uint32_t *adjrow) {
    int j;
    uint32_t l = dissect_three_join(o->k, adjrow, &j);
    int other[2], c = 0;
    for (int i = 0; i < o->k; i++) if (((l >> i) & 1u) && i != j) other[c++] = i;
    int ax = (adjrow[j] >> other[0]) & 1u, ay = (adjrow[j] >> other[1]) & 1u;
    if (ax && ay) return edge_kept(o, u[j], u[other[0]]) && edge_kept(o, u[j], u[other[1]]);
    int cen = ax ? other[0] : other[1], end = ax ? other[1] : other[0];
    return edge_kept(o, u[j], u[cen]) && edge_kept(o, u[cen], u[end]);
}

static void record(oracle_t *o, const int32_t *u, const int32_t *lab, const uint32_t *adjrow) {
    if (o->stop) return;
    if (o->budget > 0 && ++o->seen >= o->budget) o->stop = 1;
    memo_t *m = canonical(o, lab, adjrow);
    pattern_t *p = &o->pat[m->pattern];
    p->count++;
    const uint8_t *perm = o->pool + m->perm_off;
    for (int32_t q = 0; q < m->nopt; q++, perm += o->k)
        for (int c = 0; c < o->k; c++) vset_insert(&p->dom[c], u[perm[c]]);
    if (o->sampled && o->k >= 3 && kept(o, u, adjrow)) {
        p->scount++;
        perm = o->pool + m->perm_off;
        for (int32_t q = 0; q < m->nopt; q++, perm += o->k)
            for (int c = 0; c < o->k; c++) vset_insert(&p->sdom[c], u[perm[c]]);
    }
}

static void process_set(oracle_t *o, const int32_t *vs) {
    int k = o->k;
    int32_t u[OR_MAXK], lab[OR_MAXK];
    for (int i = 0; i < k; i++) u[i] = vs[i];
    /* ascending vertex order */
    for (int i = 1; i < k; i++)
        for (int j = i; j > 0 && u[j - 1] > u[j]; j--) { int32_t t = u[j]; u[j] = u[j - 1]; u[j - 1] = t; }
    for (int i = 0; i < k; i++) lab[i] = o->labels[u[i]];
    int ne = 0, ea[OR_MAXK * OR_MAXK], eb[OR_MAXK * OR_MAXK];
    uint32_t full[OR_MAXK] = {0};
    for (int i = 0; i < k; i++)
        for (int j = i + 1; j < k; j++)
            if (adjacent(o->row_ptr, o->col, u[i], u[j])) {
                ea[ne] = i; eb[ne] = j; ne++;
                full[i] |= 1u << j; full[j] |= 1u << i;
            }
    if (o->mode == 1 || k == 1) {          /* vertex-induced: the induced edge set only */
        record(o, u, lab, full);
        return;
    }
    /* edge-induced: every subset of the induced edges that spans V' connectedly */
    uint64_t nsub = 1ULL << ne;
    for (uint64_t s = 1; s < nsub; s++) {
        if (__builtin_popcountll(s) < (unsigned)(k - 1)) continue;   /* a spanning tree needs k-1 edges */
        uint32_t adjrow[OR_MAXK] = {0};
        for (int e = 0; e < ne; e++) if (s >> e & 1ULL) {
            adjrow[ea[e]] |= 1u << eb[e]; adjrow[eb[e]] |= 1u << ea[e];
        }
        if (spans_connected(k, adjrow)) record(o, u, lab, adjrow);
    }
}

/* ------------------------------------------------------------------ ESU enumeration */

static void esu_extend(oracle_t *o, int32_t *sub, int depth, const int32_t *ext, int64_t next,
                       int32_t root) {
    if (o->stop) return;
    if (depth == o->k) { process_set(o, sub); return; }
    if (next == 0) return;
    /* extension array for children: at most next - 1 + deg(w) entries */
    for (int64_t idx = next - 1; idx >= 0 && !o->stop; idx--) {
        int32_t w = ext[idx];
        int64_t deg = o->row_ptr[w + 1] - o->row_ptr[w];
        int32_t *ext2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)(idx + deg + 1));
        int64_t n2 = 0;
        for (int64_t j = 0; j < idx; j++) ext2[n2++] = ext[j];   /* Vext minus w (and minus the ones already tried) */
        for (int32_t q = o->row_ptr[w]; q < o->row_ptr[w + 1]; q++) {
            int32_t x = o->col[q];
            if (x <= root) continue;
            int excl = 1;
            for (int d = 0; d < depth && excl; d++)
                if (sub[d] == x || adjacent(o->row_ptr, o->col, sub[d], x)) excl = 0;
            if (excl) ext2[n2++] = x;
        }
        sub[depth] = w;
        esu_extend(o, sub, depth + 1, ext2, n2, root);
        free(ext2);
    }
}

/* ------------------------------------------------------------------ public entry points */

typedef struct {
    int k; int64_t npat;
    int32_t *labels;     /* npat x k */
    uint64_t *adj;       /* bit (i*k + j) set for canonical edge i < j (k <= 8; 0 for k = 9) */
    uint64_t *pairs;     /* bit q set when pair q of (0,1), (0,2), ..., (k-2,k-1) is an edge */
    int64_t *support, *count;
    int64_t *ssupport, *scount;   /* sampled mode: min_c |sampled images|, kept embeddings */
    int64_t *spop;                /* sampled mode: |sampled images of position c|, npat x k */
    double *sdeg;                 /* sampled mode: sum of log(1 + degree) over those images, npat x k */
} oracle_result_t;

static int code_sort_k;
static const pattern_t *code_sort_base;
static int idx_cmp(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return code_cmp(&code_sort_base[x].code, &code_sort_base[y].code, code_sort_k);
}

/* Unpack a canonical adjacency sequence (first pair most significant) into bit (i*k + j) of
 * *bits (k <= 8; 0 for k = 9, whose 72 bit positions do not fit) and bit q of *pairs. */
static void unpack_code(int k, uint64_t code, uint64_t *bits, uint64_t *pairs) {
    int np = k * (k - 1) / 2, idx = 0;
    uint64_t b = 0, pr = 0;
    for (int i = 0; i < k; i++)
        for (int j = i + 1; j < k; j++, idx++)
            if ((code >> (np - 1 - idx)) & 1u) {
                if (k <= 8) b |= 1ULL << (i * k + j);
                pr |= 1ULL << idx;
            }
    *bits = b;
    *pairs = pr;
}

/*
 * oracle_mine: every pattern of exactly k vertices with MNI support >= t.
 *   mode 0 = edge-induced, 1 = vertex-induced.  Only connected sets whose smallest vertex lies
 *   in [root_begin, root_end) are enumerated (the full graph: 0, n); a partial range gives a
 *   bounded sample of the work, and so does max_embeddings > 0, which stops the enumeration
 *   (roots in ascending order) after that many embeddings.  Returns NULL on bad arguments.
 */
oracle_result_t *oracle_mine_sampled(int32_t n, const int32_t *row_ptr, const int32_t *col,
                                     const int32_t *labels, int32_t k, int32_t mode, int64_t t,
                                     int32_t root_begin, int32_t root_end, int64_t max_embeddings,
                                     int32_t sampled, uint64_t seed, double p);

oracle_result_t *oracle_mine(int32_t n, const int32_t *row_ptr, const int32_t *col,
                             const int32_t *labels, int32_t k, int32_t mode, int64_t t,
                             int32_t root_begin, int32_t root_end, int64_t max_embeddings) {
    return oracle_mine_sampled(n, row_ptr, col, labels, k, mode, t, root_begin, root_end, max_embeddings,
                               0, 0, 1.0);
}

/*
 * oracle_mine_sampled: oracle_mine, plus (sampled != 0, k >= 3) the sampled statistics of
 * sampled mining at rate p: directed edges x -> y are kept when splitmix64(splitmix64(
 * splitmix64(seed) ^ x) ^ y) < floor(sqrt(p) * 2^64), and an embedding is kept when the
 * 3-vertex part of its smallest-vertex-first dissection is kept as seen from the join vertex
 * (see kept()); per pattern, ssupport = min over positions of the number of images over kept
 * embeddings (every optimal permutation) and scount = kept embeddings.
 */
oracle_result_t *oracle_mine_sampled(int32_t n, const int32_t *row_ptr, const int32_t *col,
                                     const int32_t *labels, int32_t k, int32_t mode, int64_t t,
                                     int32_t root_begin, int32_t root_end, int64_t max_embeddings,
                                     int32_t sampled, uint64_t seed, double p) {
    if (k < 1 || k > OR_MAXK || n < 0 || (mode != 0 && mode != 1)) return NULL;
    oracle_t o;
    memset(&o, 0, sizeof(o));
    o.k = k; o.mode = mode; o.row_ptr = row_ptr; o.col = col; o.labels = labels; o.n = n;
    o.budget = max_embeddings;
    o.sampled = sampled;
    o.seed = seed;
    o.thr = sampled ? (uint64_t)(sqrt(p) * 18446744073709551616.0) : 0;
    o.cx.k = k;
    gen_perms(&o.cx);
    if (root_begin < 0) root_begin = 0;
    if (root_end > n) root_end = n;
    int32_t sub[OR_MAXK];
    for (int32_t v = root_begin; v < root_end && !o.stop; v++) {
        sub[0] = v;
        int64_t deg = row_ptr[v + 1] - row_ptr[v];
        int32_t *ext = (int32_t *)malloc(sizeof(int32_t) * (size_t)(deg + 1));
        int64_t ne = 0;
        for (int32_t q = row_ptr[v]; q < row_ptr[v + 1]; q++) if (col[q] > v) ext[ne++] = col[q];
        esu_extend(&o, sub, 1, ext, ne, v);
        free(ext);
    }
    /* filter and sort */
    oracle_result_t *r = (oracle_result_t *)calloc(1, sizeof(oracle_result_t));
    r->k = k;
    int64_t *keep = (int64_t *)malloc(sizeof(int64_t) * (size_t)(o.npat + 1));
    int64_t nk = 0;
    for (int64_t p = 0; p < o.npat; p++) {
        int64_t sigma = -1;
        for (int c = 0; c < k; c++) {
            int64_t s = o.pat[p].dom[c].size;
            if (sigma < 0 || s < sigma) sigma = s;
        }
        if (sigma >= t) keep[nk++] = p;
    }
    code_sort_k = k; code_sort_base = o.pat;
    qsort(keep, (size_t)nk, sizeof(int64_t), idx_cmp);
    r->npat = nk;
    r->labels = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nk * k + 1));
    r->adj = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nk + 1));
    r->pairs = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nk + 1));
    r->support = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nk + 1));
    r->count = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nk + 1));
    r->ssupport = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nk + 1));
    r->scount = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nk + 1));
    r->spop = (int64_t *)calloc((size_t)(nk * k + 1), sizeof(int64_t));
    r->sdeg = (double *)calloc((size_t)(nk * k + 1), sizeof(double));
    for (int64_t q = 0; q < nk; q++) {
        const pattern_t *p = &o.pat[keep[q]];
        int64_t sigma = -1;
        for (int c = 0; c < k; c++) {
            int64_t s = p->dom[c].size;
            if (sigma < 0 || s < sigma) sigma = s;
        }
        for (int c = 0; c < k; c++) r->labels[q * k + c] = p->code.lab[c];
        unpack_code(k, p->code.adj, &r->adj[q], &r->pairs[q]);
        r->support[q] = sigma;
        r->count[q] = p->count;
        int64_t ss = -1;
        for (int c = 0; c < k; c++) {
            int64_t s2 = p->sdom[c].size;
            if (ss < 0 || s2 < ss) ss = s2;
        }
        r->ssupport[q] = p->scount ? ss : 0;
        r->scount[q] = p->scount;
        for (int c = 0; c < k; c++) {
            const vset_t *d = &p->sdom[c];
            r->spop[q * k + c] = d->size;
            double sd = 0.0;
            for (int64_t x = 0; x < d->cap; x++)
                if (d->slot[x] >= 0) sd += log1p((double)(row_ptr[d->slot[x] + 1] - row_ptr[d->slot[x]]));
            r->sdeg[q * k + c] = sd;
        }
    }
    free(keep);
    for (int64_t p = 0; p < o.npat; p++)
        for (int c = 0; c < OR_MAXK; c++) { free(o.pat[p].dom[c].slot); free(o.pat[p].sdom[c].slot); }
    free(o.pat); free(o.pat_slot); free(o.memo); free(o.pool); free(o.cx.perms);
    return r;
}

int64_t oracle_result_count(const oracle_result_t *r) { return r ? r->npat : -1; }

void oracle_result_copy(const oracle_result_t *r, int32_t *labels, uint64_t *adj,
                        int64_t *support, int64_t *count) {
    if (!r) return;
    memcpy(labels, r->labels, sizeof(int32_t) * (size_t)(r->npat * r->k));
    memcpy(adj, r->adj, sizeof(uint64_t) * (size_t)r->npat);
    memcpy(support, r->support, sizeof(int64_t) * (size_t)r->npat);
    memcpy(count, r->count, sizeof(int64_t) * (size_t)r->npat);
}

/* pairs[q]: bit q set when pair q of (0,1), (0,2), ..., (k-2,k-1) is a canonical edge (any k) */
void oracle_result_copy_pairs(const oracle_result_t *r, uint64_t *pairs) {
    if (!r) return;
    memcpy(pairs, r->pairs, sizeof(uint64_t) * (size_t)r->npat);
}

void oracle_result_copy_sampled(const oracle_result_t *r, int64_t *ssupport, int64_t *scount) {
    if (!r) return;
    memcpy(ssupport, r->ssupport, sizeof(int64_t) * (size_t)r->npat);
    memcpy(scount, r->scount, sizeof(int64_t) * (size_t)r->npat);
}

/* sampled mode: per pattern and canonical position, the size of the sampled image set and the
 * sum of log(1 + degree) over it (both npat x k, row-major) */
void oracle_result_copy_sampled_domains(const oracle_result_t *r, int64_t *spop, double *sdeg) {
    if (!r) return;
    memcpy(spop, r->spop, sizeof(int64_t) * (size_t)(r->npat * r->k));
    memcpy(sdeg, r->sdeg, sizeof(double) * (size_t)(r->npat * r->k));
}

void oracle_free(oracle_result_t *r) {
    if (!r) return;
    free(r->labels); free(r->adj); free(r->pairs); free(r->support); free(r->count); free(r->ssupport); free(r->scount);
    free(r->spop); free(r->sdeg); free(r);
}

/* ------------------------------------------------------------------ one pattern at a time */

/*
 * oracle_pattern_support: MNI support and embedding count of ONE pattern P in G, by matching.
 *   P has k vertices with labels plab[k] and an edge (i, j), i < j, wherever bit i*k + j of padj
 *   is set (k <= 8; oracle_pattern_support_rows takes adjacency rows instead, for any k <= 9);
 *   P must be connected.  Every injective map f from P's vertices to G's vertices that
 *   keeps labels and sends each pattern edge to a graph edge is enumerated (edge-induced mode:
 *   the monomorphisms), or that also sends each pattern non-edge to a non-edge (vertex-induced
 *   mode).  These maps are exactly the isomorphisms from P onto its embeddings, so Definition 2
 *   gives sigma = min over positions c of |{f(c)}|; each embedding is hit by |Aut(P)| maps, so
 *   the embedding count is (number of maps) / |Aut(P)|, with Aut(P) found by trying all k!
 *   vertex permutations of P.
 *   Returns 0, or -1 on bad arguments, or -2 if more than max_maps maps exist (max_maps > 0).
 * Independent of oracle_mine: no ESU, no canonical form.
 */
typedef struct {
    int k, mode;
    const int32_t *row_ptr, *col, *labels;
    int32_t n;
    int32_t plab[OR_MAXK];
    uint32_t padj[OR_MAXK];
    int order[OR_MAXK], parent[OR_MAXK];
    int32_t f[OR_MAXK];
    uint8_t **img;               /* per position: bitmap over n */
    int64_t maps, max_maps;
    int over;
} match_t;

static void match_rec(match_t *m, int depth) {
    if (m->over) return;
    if (depth == m->k) {
        m->maps++;
        if (m->max_maps > 0 && m->maps > m->max_maps) { m->over = 1; return; }
        for (int c = 0; c < m->k; c++) m->img[c][m->f[c] >> 3] |= (uint8_t)(1u << (m->f[c] & 7));
        return;
    }
    int c = m->order[depth];
    int32_t lo, hi;
    const int32_t *cand;
    int32_t all_first = 0;
    if (depth == 0) { lo = 0; hi = m->n; cand = NULL; all_first = 1; }
    else { int32_t pv = m->f[m->parent[depth]]; lo = m->row_ptr[pv]; hi = m->row_ptr[pv + 1]; cand = m->col; }
    for (int32_t q = lo; q < hi && !m->over; q++) {
        int32_t x = all_first ? q : cand[q];
        if (m->labels[x] != m->plab[c]) continue;
        int ok = 1;
        for (int e = 0; e < depth && ok; e++) {
            int c2 = m->order[e];
            if (m->f[c2] == x) { ok = 0; break; }
            int pe = (m->padj[c] >> c2) & 1u;
            if (pe && !adjacent(m->row_ptr, m->col, x, m->f[c2])) ok = 0;
            if (!pe && m->mode == 1 && adjacent(m->row_ptr, m->col, x, m->f[c2])) ok = 0;
        }
        if (!ok) continue;
        m->f[c] = x;
        match_rec(m, depth + 1);
    }
}

/* The same with P's adjacency given as rows: bit j of prow[i] set for every edge (i, j) (any
 * k <= 9; the rows must be symmetric and without self-loops). */
int oracle_pattern_support_rows(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *labels,
                                int32_t k, const int32_t *plab, const uint32_t *prow, int32_t mode,
                                int64_t max_maps, int64_t *support, int64_t *count) {
    if (k < 1 || k > OR_MAXK || n < 1 || (mode != 0 && mode != 1) || !support || !count || !prow) return -1;
    match_t m;
    memset(&m, 0, sizeof(m));
    m.k = k; m.mode = mode; m.row_ptr = row_ptr; m.col = col; m.labels = labels; m.n = n;
    m.max_maps = max_maps;
    for (int i = 0; i < k; i++) m.plab[i] = plab[i];
    for (int i = 0; i < k; i++) {
        if ((prow[i] >> i) & 1u) return -1;
        for (int j = 0; j < k; j++)
            if (((prow[i] >> j) & 1u) != ((prow[j] >> i) & 1u)) return -1;
        m.padj[i] = prow[i] & ((1u << k) - 1u);
    }
    if (!spans_connected(k, m.padj)) return -1;
    /* BFS order from position 0: each later position has an already placed neighbour */
    int seen = 1; m.order[0] = 0; m.parent[0] = -1;
    for (int d = 0, tail = 1; d < tail; d++) {
        int c = m.order[d];
        for (int x = 0; x < k; x++)
            if (!((seen >> x) & 1) && ((m.padj[c] >> x) & 1u)) {
                seen |= 1 << x; m.order[tail] = x; m.parent[tail] = d; tail++;
            }
    }
    /* parent[] holds the index in order[]; convert to the position itself */
    for (int d = 1; d < k; d++) m.parent[d] = m.order[m.parent[d]];
    m.img = (uint8_t **)malloc(sizeof(uint8_t *) * (size_t)k);
    for (int c = 0; c < k; c++) m.img[c] = (uint8_t *)calloc((size_t)n / 8 + 1, 1);
    match_rec(&m, 0);
    int rc = 0;
    if (m.over) rc = -2;
    else {
        int64_t sigma = -1;
        for (int c = 0; c < k; c++) {
            int64_t s = 0;
            for (int32_t b = 0; b < n / 8 + 1; b++) s += __builtin_popcount(m.img[c][b]);
            if (sigma < 0 || s < sigma) sigma = s;
        }
        /* automorphisms: label- and adjacency-preserving permutations of P */
        canon_ctx_t cx;
        memset(&cx, 0, sizeof(cx));
        cx.k = k;
        gen_perms(&cx);
        int64_t aut = 0;
        for (int p = 0; p < cx.nperm; p++) {
            const uint8_t *pi = cx.perms + (size_t)p * k;
            int ok = 1;
            for (int i = 0; i < k && ok; i++) {
                if (m.plab[pi[i]] != m.plab[i]) ok = 0;
                for (int j = 0; j < k && ok; j++)
                    if ((((m.padj[i] >> j) & 1u)) != ((m.padj[pi[i]] >> pi[j]) & 1u)) ok = 0;
            }
            aut += ok;
        }
        free(cx.perms);
        *support = m.maps ? sigma : 0;
        *count = m.maps / aut;
    }
    for (int c = 0; c < k; c++) free(m.img[c]);
    free(m.img);
    return rc;
}

int oracle_pattern_support(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *labels,
                           int32_t k, const int32_t *plab, uint64_t padj_bits, int32_t mode,
                           int64_t max_maps, int64_t *support, int64_t *count) {
    if (k < 1 || k > 8) return -1;      /* bit (i*k + j) runs past 64 bits at k = 9 */
    uint32_t prow[OR_MAXK] = {0};
    for (int i = 0; i < k; i++)
        for (int j = i + 1; j < k; j++)
            if ((padj_bits >> (i * k + j)) & 1ULL) { prow[i] |= 1u << j; prow[j] |= 1u << i; }
    return oracle_pattern_support_rows(n, row_ptr, col, labels, k, plab, prow, mode, max_maps, support, count);
}

/* dissection of a connected k-vertex graph given as adjacency rows over positions 0..k-1
 * (positions are the ids); returns the 3-vertex part as a mask, 0 if none */
uint32_t oracle_dissect(int32_t k, const uint32_t *adjrow) {
    if (k < 3 || k > OR_MAXK) return 0;
    return dissect_three(k, adjrow);
}

/* Test hooks (the pins call these directly):
 *   oracle_dissect_join  the dissection of a connected graph on positions 0..k-1 (positions are
 *                        the ids): 3-vertex part as a mask, its join vertex in *join;
 *   oracle_edge_kept     the sampling rule of one directed edge x -> y at rate p (kept at rate
 *                        sqrt(p), so a 3-vertex part made of two kept edges survives at rate p);
 *   oracle_kept          whether an embedding (vertex ids u[0..k) ascending, adjacency rows
 *                        over positions) is kept by sampled mining at rate p. */
uint32_t oracle_dissect_join(int32_t k, const uint32_t *adjrow, int32_t *join) {
    int j = -1;
    uint32_t l = (k >= 3 && k <= OR_MAXK) ? dissect_three_join(k, adjrow, &j) : 0;
    *join = j;
    return l;
}

int oracle_edge_kept(uint64_t seed, double p, int32_t x, int32_t y) {
    oracle_t o;
    memset(&o, 0, sizeof(o));
    o.seed = seed;
    o.thr = (uint64_t)(sqrt(p) * 18446744073709551616.0);
    return edge_kept(&o, x, y);
}

int oracle_kept(int32_t k, const int32_t *u, const uint32_t *adjrow, uint64_t seed, double p) {
    if (k < 3 || k > OR_MAXK) return -1;
    oracle_t o;
    memset(&o, 0, sizeof(o));
    o.k = k;
    o.seed = seed;
    o.thr = (uint64_t)(sqrt(p) * 18446744073709551616.0);
    return kept(&o, u, adjrow);
}

/* ================================================================== quota-sampled mining
 *
 * Section 5's subgraph sampling with fixed iteration counts, taken through the method's own
 * steps (an approximation has no plain definition to compute), slowly and directly:
 *   1. size 1: the frequent labels;
 *   2. size 3 ("matching"): every vertex v with a frequent label runs its candidate pieces
 *      (numbered as below), at most match_quota of them when match_quota > 0; a candidate
 *      becomes a size-3 embedding only if v is its smallest vertex;
 *   3. even k: size 2, every edge, exactly;
 *   4. joins l -> l+2: every stored frequent size-l embedding s and every vertex v of s (the
 *      key group of v) runs the candidate pieces keyed at v -- at most join_quota^2 of them --
 *      and, when l = 2, only join_quota edges per key vertex are joined; each candidate piece t
 *      (disjoint from s but for v, of a frequent size-3 pattern) is joined with every subset of
 *      the cross edges (edge-induced) or all of them (vertex-induced), pruned when a connected
 *      triple {v, s[p], t[q]} has an infrequent size-3 pattern (Section 4.5), and kept when the
 *      smallest-vertex-first dissection of the result returns exactly (t, v) (Algorithm 1);
 *   5. every level keeps the embeddings of patterns whose MNI support over the drawn
 *      embeddings reaches t; the last level's patterns are the output.
 * Candidate pieces of key vertex v with neighbour list N (length d): first the centre pairs
 * {N[x], N[y]}, x < y, numbered y(y-1)/2 + x -- except when joining an edge {v, w}, where only
 * pairs with x < c, c = |{z in N : z < w}|, are candidates (the others never survive the
 * dissection): rows y < c numbered as before, then row y >= c, column x at
 * c(c-1)/2 + (y - c) c + x -- then the end pieces v - a - b, a = N[j], b = N(a)[r], numbered
 * (sum of d(N[j']) over j' < j) + r.  A centre pair is a wedge centred at v, plus (edge-induced)
 * a triangle when a ~ b, or (vertex-induced) only that triangle; an end piece is the wedge
 * centred at a (none when b = v, or vertex-induced when b ~ v).
 * Draws: a unit with c candidates and quota Q < c runs candidates (a j + b) mod c, j < Q, with
 * h = H(... H(H(seed) ^ x_0) ... ^ x_{l-1}) then H(h ^ (2^32 + v)) over the ascending ids x of
 * s (H = one splitmix64 step), a = the first integer coprime to c at or after 1 + (h mod (c-1))
 * (wrapping from c - 1 to 1), b = H(h) mod c; an edge {v, w} at position pos of v's list runs
 * when d(v) <= X or (a_v pos + b_v) mod d(v) < X, (a_v, b_v) drawn likewise from
 * H(H(seed) ^ (2^33 + v)) with modulus d(v). */

static uint64_t q_gcd(uint64_t x, uint64_t y) { while (y) { uint64_t r = x % y; x = y; y = r; } return x; }

static void q_draw(uint64_t h, uint64_t c, uint64_t *a, uint64_t *b) {
    uint64_t x = 1 + h % (c - 1);
    while (q_gcd(x, c) != 1) x = (x + 1 == c) ? 1 : x + 1;
    *a = x;
    *b = smix(h) % c;
}

typedef struct { int l; int64_t n, cap; int32_t *v; uint32_t *adj; int32_t *pat; } estore_t;

static void es_push(estore_t *e, const int32_t *v, const uint32_t *adj, int32_t pat) {
    if (e->n == e->cap) {
        e->cap = e->cap ? e->cap * 2 : 1024;
        e->v = (int32_t *)realloc(e->v, sizeof(int32_t) * (size_t)(e->cap * e->l));
        e->adj = (uint32_t *)realloc(e->adj, sizeof(uint32_t) * (size_t)(e->cap * e->l));
        e->pat = (int32_t *)realloc(e->pat, sizeof(int32_t) * (size_t)e->cap);
    }
    memcpy(e->v + e->n * e->l, v, sizeof(int32_t) * (size_t)e->l);
    memcpy(e->adj + e->n * e->l, adj, sizeof(uint32_t) * (size_t)e->l);
    e->pat[e->n++] = pat;
}

static void es_free(estore_t *e) { free(e->v); free(e->adj); free(e->pat); }

static void q_ctx_init(oracle_t *o, int k, const int32_t *row_ptr, const int32_t *col, const int32_t *labels,
                       int32_t n, int mode) {
    memset(o, 0, sizeof(*o));
    o->k = k; o->mode = mode; o->row_ptr = row_ptr; o->col = col; o->labels = labels; o->n = n;
    o->cx.k = k;
    gen_perms(&o->cx);
}

static void q_ctx_free(oracle_t *o) {
    for (int64_t p = 0; p < o->npat; p++)
        for (int c = 0; c < OR_MAXK; c++) { free(o->pat[p].dom[c].slot); free(o->pat[p].sdom[c].slot); }
    free(o->pat); free(o->pat_slot); free(o->memo); free(o->pool); free(o->cx.perms);
}

/* record one embedding (vertex ids u in any order, adjacency rows over the same positions):
 * its pattern, count and images; returns the pattern index */
static int32_t q_record(oracle_t *o, const int32_t *u, const uint32_t *adjrow) {
    int32_t lab[OR_MAXK];
    for (int i = 0; i < o->k; i++) lab[i] = o->labels[u[i]];
    memo_t *m = canonical(o, lab, adjrow);
    pattern_t *p = &o->pat[m->pattern];
    p->count++;
    const uint8_t *perm = o->pool + m->perm_off;
    for (int32_t q = 0; q < m->nopt; q++, perm += o->k)
        for (int c = 0; c < o->k; c++) vset_insert(&p->dom[c], u[perm[c]]);
    return m->pattern;
}

static int64_t q_sigma(const pattern_t *p, int k) {
    int64_t s = -1;
    for (int c = 0; c < k; c++) if (s < 0 || p->dom[c].size < s) s = p->dom[c].size;
    return s;
}

/* embeddings of the patterns of o with support >= t (positions ascending by id) */
static void q_keep_frequent(const oracle_t *o, const estore_t *all, int64_t t, estore_t *out) {
    out->l = all->l;
    for (int64_t e = 0; e < all->n; e++)
        if (q_sigma(&o->pat[all->pat[e]], o->k) >= t) es_push(out, all->v + e * all->l, all->adj + e * all->l, all->pat[e]);
}

/* is the size-3 graph (ids u, rows adj over 3 positions) of a frequent size-3 pattern of o3? */
static int q_frequent3(oracle_t *o3, const int32_t *u, const uint32_t *adj, int64_t t) {
    int32_t lab[3] = {o3->labels[u[0]], o3->labels[u[1]], o3->labels[u[2]]};
    memo_t *m = canonical(o3, lab, adj);
    return q_sigma(&o3->pat[m->pattern], 3) >= t;
}

/* decode candidate idx of key vertex v (list N, length d); cpos >= 0: joining the edge {v, w}
 * with cpos entries of N below w.  Returns 1 for a centre pair, 0 for an end piece. */
static int q_decode(const int32_t *row_ptr, const int32_t *col, int32_t v, int64_t idx, int64_t cpos, int32_t *a,
                    int32_t *b) {
    const int32_t *N = col + row_ptr[v];
    const int64_t d = row_ptr[v + 1] - row_ptr[v];
    const int64_t tri = cpos >= 0 ? cpos * (cpos - 1) / 2 : d * (d - 1) / 2;
    const int64_t nc = cpos >= 0 ? tri + (d - cpos) * cpos : tri;
    if (idx < nc) {
        int64_t x, y;
        if (idx < tri) {
            y = 1;
            while ((y + 1) * y / 2 <= idx) y++;
            x = idx - y * (y - 1) / 2;
        } else {
            const int64_t r = idx - tri;
            y = cpos + r / cpos;
            x = r % cpos;
        }
        *a = N[x]; *b = N[y];
        return 1;
    }
    int64_t r = idx - nc;
    for (int64_t j = 0; j < d; j++) {
        const int64_t dj = row_ptr[N[j] + 1] - row_ptr[N[j]];
        if (r < dj) { *a = N[j]; *b = col[row_ptr[N[j]] + r]; return 0; }
        r -= dj;
    }
    *a = *b = -1;
    return 0;
}

static int q_pos_of(const int32_t *u, int l, int32_t x) {
    for (int i = 0; i < l; i++) if (u[i] == x) return i;
    return -1;
}

/* one join level: s (size l) -> next (size l+2), recorded in o (k = l+2) and stored in all */
static void q_join(oracle_t *o, oracle_t *o3, int64_t t, const estore_t *s, uint64_t seed, int64_t X, estore_t *all) {
    const int l = s->l, K = l + 2;
    const int32_t *row_ptr = o->row_ptr, *col = o->col;
    const int64_t Q = X * X;
    all->l = K;
    for (int64_t e = 0; e < s->n; e++) {
        const int32_t *u = s->v + e * l;      /* ascending ids */
        const uint32_t *sa = s->adj + e * l;
        for (int i = 0; i < l; i++) {
            const int32_t v = u[i];
            const int64_t d = row_ptr[v + 1] - row_ptr[v];
            int64_t cpos = -1;
            if (l == 2) {
                const int32_t w = u[1 - i];
                cpos = 0;
                while (cpos < d && col[row_ptr[v] + cpos] < w) cpos++;
                if (X > 0 && d > X) {   /* edge quota of the key vertex */
                    uint64_t av, bv;
                    q_draw(smix(smix(seed) ^ ((1ULL << 33) + (uint64_t)(uint32_t)v)), (uint64_t)d, &av, &bv);
                    if ((av * (uint64_t)cpos + bv) % (uint64_t)d >= (uint64_t)X) continue;
                }
            }
            int64_t c = cpos >= 0 ? cpos * (cpos - 1) / 2 + (d - cpos) * cpos : d * (d - 1) / 2;
            for (int64_t j = 0; j < d; j++) { int32_t a = col[row_ptr[v] + j]; c += row_ptr[a + 1] - row_ptr[a]; }
            uint64_t qa = 1, qb = 0;
            int64_t runs = c;
            if (Q > 0 && c > Q) {
                uint64_t h = smix(seed);
                for (int q = 0; q < l; q++) h = smix(h ^ (uint64_t)(uint32_t)u[q]);
                h = smix(h ^ ((1ULL << 32) + (uint64_t)(uint32_t)v));
                q_draw(h, (uint64_t)c, &qa, &qb);
                runs = Q;
            }
            for (int64_t jj = 0; jj < runs; jj++) {
                const int64_t idx = runs == c ? jj : (int64_t)((qa * (uint64_t)jj + qb) % (uint64_t)c);
                int32_t a, b;
                const int centre = q_decode(row_ptr, col, v, idx, cpos, &a, &b);
                if (a < 0 || b == v || q_pos_of(u, l, a) >= 0 || q_pos_of(u, l, b) >= 0) continue;
                const int closed = adjacent(row_ptr, col, a, b);
                /* the piece's edge sets over (v, a, b): bit 0 v-a, bit 1 v-b, bit 2 a-b */
                int shapes[2], ns = 0;
                if (centre) {
                    if (o->mode == 1) shapes[ns++] = closed ? 7 : 3;
                    else { shapes[ns++] = 3; if (closed) shapes[ns++] = 7; }
                } else {
                    if (o->mode == 1 && adjacent(row_ptr, col, v, b)) continue;
                    shapes[ns++] = 5;
                }
                for (int si = 0; si < ns; si++) {
                    const int sh = shapes[si];
                    /* the piece's own pattern must be frequent */
                    int32_t pu[3] = {v, a, b};
                    uint32_t pr[3] = {0, 0, 0};
                    if (sh & 1) { pr[0] |= 2; pr[1] |= 1; }
                    if (sh & 2) { pr[0] |= 4; pr[2] |= 1; }
                    if (sh & 4) { pr[1] |= 4; pr[2] |= 2; }
                    if (!q_frequent3(o3, pu, pr, t)) continue;
                    /* cross edges between s \ {v} and {a, b} */
                    int cp[2 * OR_MAXK], cx[2 * OR_MAXK], nav = 0;
                    for (int p = 0; p < l; p++) {
                        if (p == i) continue;
                        if (adjacent(row_ptr, col, u[p], a)) { cp[nav] = p; cx[nav] = 0; nav++; }
                        if (adjacent(row_ptr, col, u[p], b)) { cp[nav] = p; cx[nav] = 1; nav++; }
                    }
                    const uint32_t full = (1u << nav) - 1u;
                    for (uint32_t sub = (o->mode == 1 ? full : 0);; sub++) {
                        /* joining-point pruning */
                        int pruned = 0;
                        for (int p = 0; p < l && !pruned; p++) {
                            if (p == i) continue;
                            for (int q = 0; q < 2 && !pruned; q++) {
                                const int32_t xq = q ? b : a;
                                const int e1 = (sa[i] >> p) & 1u;
                                const int e2 = q ? ((sh >> 1) & 1) : (sh & 1);
                                int e3 = 0;
                                for (int z = 0; z < nav; z++) if (((sub >> z) & 1u) && cp[z] == p && cx[z] == q) e3 = 1;
                                if (e1 + e2 + e3 < 2) continue;
                                int32_t tu[3] = {v, u[p], xq};
                                uint32_t tr[3] = {0, 0, 0};
                                if (e1) { tr[0] |= 2; tr[1] |= 1; }
                                if (e2) { tr[0] |= 4; tr[2] |= 1; }
                                if (e3) { tr[1] |= 4; tr[2] |= 2; }
                                if (!q_frequent3(o3, tu, tr, t)) pruned = 1;
                            }
                        }
                        if (!pruned) {
                            /* the joined subgraph, positions ascending by id */
                            int32_t ids[OR_MAXK];
                            for (int p = 0; p < l; p++) ids[p] = u[p];
                            ids[l] = a; ids[l + 1] = b;
                            uint32_t rows[OR_MAXK] = {0};
                            for (int p = 0; p < l; p++) rows[p] = sa[p];
                            if (sh & 1) { rows[i] |= 1u << l; rows[l] |= 1u << i; }
                            if (sh & 2) { rows[i] |= 1u << (l + 1); rows[l + 1] |= 1u << i; }
                            if (sh & 4) { rows[l] |= 1u << (l + 1); rows[l + 1] |= 1u << l; }
                            for (int z = 0; z < nav; z++)
                                if ((sub >> z) & 1u) {
                                    const int h2 = l + cx[z];
                                    rows[cp[z]] |= 1u << h2; rows[h2] |= 1u << cp[z];
                                }
                            int ord[OR_MAXK];
                            for (int h = 0; h < K; h++) ord[h] = h;
                            for (int x = 1; x < K; x++)
                                for (int y = x; y > 0 && ids[ord[y - 1]] > ids[ord[y]]; y--) { int tt = ord[y]; ord[y] = ord[y - 1]; ord[y - 1] = tt; }
                            int at[OR_MAXK];
                            for (int h = 0; h < K; h++) at[ord[h]] = h;
                            int32_t su[OR_MAXK];
                            uint32_t srow[OR_MAXK] = {0};
                            for (int h = 0; h < K; h++) {
                                su[at[h]] = ids[h];
                                for (int h2 = 0; h2 < K; h2++) if ((rows[h] >> h2) & 1u) srow[at[h]] |= 1u << at[h2];
                            }
                            int jn;
                            const uint32_t lm = dissect_three_join(K, srow, &jn);
                            const uint32_t want = (1u << at[i]) | (1u << at[l]) | (1u << at[l + 1]);
                            if (lm == want && jn == at[i]) {
                                const int32_t pat = q_record(o, su, srow);
                                es_push(all, su, srow, pat);
                            }
                        }
                        if (o->mode == 1 || sub == full) break;
                    }
                }
            }
        }
    }
}

static oracle_result_t *q_result(const oracle_t *o, int k, int64_t t) {
    oracle_result_t *r = (oracle_result_t *)calloc(1, sizeof(oracle_result_t));
    r->k = k;
    int64_t *keep = (int64_t *)malloc(sizeof(int64_t) * (size_t)(o->npat + 1));
    int64_t nk = 0;
    for (int64_t p = 0; p < o->npat; p++) if (q_sigma(&o->pat[p], k) >= t) keep[nk++] = p;
    code_sort_k = k; code_sort_base = o->pat;
    qsort(keep, (size_t)nk, sizeof(int64_t), idx_cmp);
    r->npat = nk;
    r->labels = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nk * k + 1));
    r->adj = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nk + 1));
    r->pairs = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nk + 1));
    r->support = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nk + 1));
    r->count = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nk + 1));
    for (int64_t q = 0; q < nk; q++) {
        const pattern_t *p = &o->pat[keep[q]];
        for (int c = 0; c < k; c++) r->labels[q * k + c] = p->code.lab[c];
        unpack_code(k, p->code.adj, &r->adj[q], &r->pairs[q]);
        r->support[q] = q_sigma(p, k);
        r->count[q] = p->count;
    }
    free(keep);
    return r;
}

/*
 * oracle_mine_quota: the patterns of exactly k vertices (3 <= k <= 9) whose MNI support over
 * the embeddings drawn under Section 5's quotas reaches t, with those supports and counts (see
 * the steps above).  join_quota = 0 and match_quota = 0 draw everything, which is exact mining
 * by the method's own steps.
 */
oracle_result_t *oracle_mine_quota(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *labels,
                                   int32_t k, int32_t mode, int64_t t, uint64_t seed, int64_t join_quota,
                                   int64_t match_quota) {
    if (k < 3 || k > OR_MAXK || n < 0 || (mode != 0 && mode != 1) || join_quota < 0 || match_quota < 0) return NULL;
    int64_t cls[256] = {0};
    for (int32_t v = 0; v < n; v++) cls[labels[v] & 0xff]++;
    /* size 3 by matching from each vertex with a frequent label */
    oracle_t o3;
    q_ctx_init(&o3, 3, row_ptr, col, labels, n, mode);
    estore_t all3 = {3, 0, 0, NULL, NULL, NULL};
    for (int32_t v = 0; v < n; v++) {
        if (cls[labels[v] & 0xff] < t) continue;
        const int64_t d = row_ptr[v + 1] - row_ptr[v];
        int64_t c = d * (d - 1) / 2;
        for (int64_t j = 0; j < d; j++) { int32_t a = col[row_ptr[v] + j]; c += row_ptr[a + 1] - row_ptr[a]; }
        uint64_t qa = 1, qb = 0;
        int64_t runs = c;
        if (match_quota > 0 && c > match_quota) {
            uint64_t h = smix(smix(seed) ^ (uint64_t)(uint32_t)v);
            h = smix(h ^ ((1ULL << 32) + (uint64_t)(uint32_t)v));
            q_draw(h, (uint64_t)c, &qa, &qb);
            runs = match_quota;
        }
        for (int64_t jj = 0; jj < runs; jj++) {
            const int64_t idx = runs == c ? jj : (int64_t)((qa * (uint64_t)jj + qb) % (uint64_t)c);
            int32_t a, b;
            const int centre = q_decode(row_ptr, col, v, idx, -1, &a, &b);
            if (b == v || a < v || b < v) continue;   /* keyed at its smallest vertex */
            const int closed = adjacent(row_ptr, col, a, b);
            int shapes[2], ns = 0;
            if (centre) {
                if (mode == 1) shapes[ns++] = closed ? 7 : 3;
                else { shapes[ns++] = 3; if (closed) shapes[ns++] = 7; }
            } else {
                if (mode == 1 && adjacent(row_ptr, col, v, b)) continue;
                shapes[ns++] = 5;
            }
            for (int si = 0; si < ns; si++) {
                const int sh = shapes[si];
                int32_t ids[3] = {v, a, b};
                uint32_t rows[3] = {0, 0, 0};
                if (sh & 1) { rows[0] |= 2; rows[1] |= 1; }
                if (sh & 2) { rows[0] |= 4; rows[2] |= 1; }
                if (sh & 4) { rows[1] |= 4; rows[2] |= 2; }
                /* ascending ids: v is the smallest; order a, b */
                if (ids[1] > ids[2]) {
                    int32_t ti = ids[1]; ids[1] = ids[2]; ids[2] = ti;
                    uint32_t r0 = rows[0], r1 = rows[1], r2 = rows[2];
                    uint32_t sw[3];
                    sw[0] = (r0 & 1u) | ((r0 >> 1) & 2u) | ((r0 << 1) & 4u);
                    sw[1] = (r2 & 1u) | ((r2 >> 1) & 2u) | ((r2 << 1) & 4u);
                    sw[2] = (r1 & 1u) | ((r1 >> 1) & 2u) | ((r1 << 1) & 4u);
                    rows[0] = sw[0]; rows[1] = sw[1]; rows[2] = sw[2];
                }
                const int32_t pat = q_record(&o3, ids, rows);
                es_push(&all3, ids, rows, pat);
            }
        }
    }
    estore_t cur = {3, 0, 0, NULL, NULL, NULL};
    oracle_t last;
    int have_last = 0;
    if (k == 3) {
        last = o3; have_last = 1;
    } else {
        if (k & 1) {
            q_keep_frequent(&o3, &all3, t, &cur);
        } else {
            /* size 2: every edge, exactly */
            oracle_t o2;
            q_ctx_init(&o2, 2, row_ptr, col, labels, n, mode);
            estore_t all2 = {2, 0, 0, NULL, NULL, NULL};
            for (int32_t x = 0; x < n; x++)
                for (int32_t q = row_ptr[x]; q < row_ptr[x + 1]; q++) {
                    if (col[q] <= x) continue;
                    int32_t ids[2] = {x, col[q]};
                    uint32_t rows[2] = {2u, 1u};
                    es_push(&all2, ids, rows, q_record(&o2, ids, rows));
                }
            cur.l = 2;
            q_keep_frequent(&o2, &all2, t, &cur);
            es_free(&all2);
            q_ctx_free(&o2);
        }
        while (cur.l + 2 <= k) {
            oracle_t on;
            q_ctx_init(&on, cur.l + 2, row_ptr, col, labels, n, mode);
            estore_t alln = {cur.l + 2, 0, 0, NULL, NULL, NULL};
            q_join(&on, &o3, t, &cur, seed, join_quota, &alln);
            es_free(&cur);
            memset(&cur, 0, sizeof(cur));
            if (alln.l == k) {
                last = on; have_last = 1;
                es_free(&alln);
                break;
            }
            q_keep_frequent(&on, &alln, t, &cur);
            es_free(&alln);
            q_ctx_free(&on);
        }
    }
    es_free(&all3);
    es_free(&cur);
    oracle_result_t *r = have_last ? q_result(&last, k, t) : NULL;
    if (have_last && k != 3) q_ctx_free(&last);
    q_ctx_free(&o3);
    return r;
}

/* test hook: the draw's (a, b) for hash h and modulus c >= 2 */
void oracle_quota_draw(uint64_t h, uint64_t c, uint64_t *a, uint64_t *b) { q_draw(h, c, a, b); }
