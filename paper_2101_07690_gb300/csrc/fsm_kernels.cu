// fsm_kernels.cu -- graph preparation, scans, quick-pattern bookkeeping, canonicalisation,
// orbits, MNI domains and supports, and the size-1 / size-2 base levels.
#include "fsm_kernels.cuh"
#include "fsm_canon.cuh"

#include <climits>

#include <atomic>

namespace fsm {

static std::atomic<int64_t> g_launches{0};
int64_t launches_so_far() { return g_launches.load(); }
void note_launches(int64_t n) { g_launches.fetch_add(n); }
#define LAUNCHED(n) note_launches(n)

namespace {

constexpr int kThreads = 256;

inline int blocks_for(int64_t n, int threads = kThreads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;   // grid-stride beyond this
    return (int)b;
}

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

// ------------------------------------------------------------------ graph preparation

__global__ void validate_kernel(DevGraph g, int32_t num_labels, int *err) {
    for (int64_t v = gtid(); v < g.n; v += gstride()) {
        const int32_t rb = g.row_ptr[v], re = g.row_ptr[v + 1];
        const int32_t lab = g.labels[v];
        bool bad = rb > re || rb < 0 || (int64_t)re > g.nnz || lab < 0 || lab >= num_labels || (v == 0 && rb != 0);
        if (!bad) {
            for (int32_t j = rb; j < re && !bad; ++j) {
                const int32_t w = g.col[j];
                if (w < 0 || w >= g.n || w == (int32_t)v || (j > rb && g.col[j - 1] >= w)) { bad = true; break; }
                // w's row is searched below: its bounds must be sane before any col read
                const int32_t wb = g.row_ptr[w], we = g.row_ptr[w + 1];
                if (wb < 0 || wb > we || (int64_t)we > g.nnz) { bad = true; break; }
                // symmetry: v must appear in N(w)
                int32_t lo = wb, hi = we;
                while (lo < hi) {
                    const int32_t mid = (lo + hi) >> 1;
                    if (g.col[mid] < (int32_t)v) lo = mid + 1; else hi = mid;
                }
                if (lo >= we || g.col[lo] != (int32_t)v) bad = true;
            }
        }
        if (bad) atomicOr(err, FSM_ERR_CSR);
    }
}

__global__ void prepare_kernel(DevGraph g, int64_t *piece_cnt, int32_t *end_off, int32_t *rank,
                               int32_t *cls_size) {
    for (int64_t v = gtid(); v < g.n; v += gstride()) {
        const int32_t rb = g.row_ptr[v], re = g.row_ptr[v + 1];
        const int64_t d = re - rb;
        int64_t run = 0;
        for (int32_t j = rb; j < re; ++j) {
            end_off[j] = (int32_t)run;
            const int32_t a = g.col[j];
            run += g.row_ptr[a + 1] - g.row_ptr[a];
        }
        piece_cnt[v] = d * (d - 1) / 2 + run;
        rank[v] = atomicAdd(cls_size + g.labels[v], 1);
    }
}

// Neighbour-adjacency matrices (see DevGraph::tri_off).  Words per vertex: d * ceil(d / 32) for
// d >= dmin, else 0.
__global__ void tri_words_kernel(DevGraph g, int32_t dmin, int64_t *words) {
    for (int64_t v = gtid(); v < g.n; v += gstride()) {
        const int64_t d = g.row_ptr[v + 1] - g.row_ptr[v];
        words[v] = d >= dmin ? d * ((d + 31) / 32) : 0;
    }
}
// One warp per vertex with a matrix: for its x-th neighbour a, every neighbour c of a that is
// also the y-th neighbour of v (y > x, found by binary search in v's sorted list) sets bit
// (x, y).
__global__ void tri_bits_kernel(DevGraph g, int32_t dmin, const int64_t *off, int64_t *tri_off, uint32_t *bits) {
    const int lane = threadIdx.x & 31;
    for (int64_t v = gtid() >> 5; v < g.n; v += gstride() >> 5) {
        const int32_t rv = g.row_ptr[v], d = g.row_ptr[v + 1] - rv;
        if (d < dmin) {
            if (lane == 0) tri_off[v] = -1;
            continue;
        }
        const int64_t base = off[v];
        const int32_t stride = (d + 31) >> 5;
        if (lane == 0) tri_off[v] = base;
        for (int32_t x = 0; x + 1 < d; ++x) {
            const int32_t a = g.col[rv + x];
            const int32_t ra = g.row_ptr[a], da = g.row_ptr[a + 1] - ra;
            for (int32_t j = lane; j < da; j += 32) {
                const int32_t c = g.col[ra + j];
                const int32_t y = count_below(g.col + rv, d, c);
                if (y > x && y < d && g.col[rv + y] == c)
                    atomicOr(bits + base + (int64_t)x * stride + (y >> 5), 1u << (y & 31));
            }
        }
    }
}

// ------------------------------------------------------------------ scan (exclusive, int64)

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int64_t kScanTile = (int64_t)kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t x, int64_t *warp_tot, int64_t &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int64_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
        int64_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        warp_tot[lane] = ti - t;          // exclusive prefix of warp totals
        if (lane == 31) warp_tot[32] = ti;
    }
    __syncthreads();
    const int64_t res = warp_tot[wid] + incl - x;
    total = warp_tot[32];
    __syncthreads();
    return res;
}

// out[i] = exclusive prefix within the tile + base[tile] (base may be NULL)
__global__ void __launch_bounds__(kScanThreads) scan_tile_kernel(const int64_t *in, int64_t *out, int64_t n,
                                                                 const int64_t *base, int64_t *tile_sum,
                                                                 bool write_total) {
    __shared__ int64_t warp_tot[33];
    const int64_t t0 = (int64_t)blockIdx.x * kScanTile;
    const int64_t i0 = t0 + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (i0 + k < n) ? in[i0 + k] : 0;
        s += v[k];
    }
    int64_t total;
    int64_t ex = block_exclusive_scan(s, warp_tot, total);
    if (out) {
        const int64_t b = base ? base[blockIdx.x] : 0;
        int64_t run = b + ex;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (i0 + k < n) out[i0 + k] = run;
            run += v[k];
        }
        if (write_total && threadIdx.x == 0 && blockIdx.x == gridDim.x - 1) out[n] = b + total;
    }
    if (tile_sum && threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

} // namespace

size_t scan_temp_bytes(int64_t n) {
    if (n <= kScanTile) return 0;
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    return (size_t)(2 * nb + 1) * sizeof(int64_t) + scan_temp_bytes(nb);
}

cudaError_t launch_scan_i64(const int64_t *in, int64_t *out, int64_t n, void *temp, cudaStream_t st) {
    if (n <= 0) {
        return cudaMemsetAsync(out, 0, sizeof(int64_t), st);
    }
    if (n <= kScanTile) {
        LAUNCHED(1);
        scan_tile_kernel<<<1, kScanThreads, 0, st>>>(in, out, n, nullptr, nullptr, true);
        return cudaGetLastError();
    }
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    int64_t *sums = (int64_t *)temp;
    int64_t *sums_x = sums + nb;
    void *rest = sums_x + nb + 1;
    LAUNCHED(1);
    scan_tile_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(in, nullptr, n, nullptr, sums, false);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_scan_i64(sums, sums_x, nb, rest, st);
    if (e != cudaSuccess) return e;
    LAUNCHED(1);
    scan_tile_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, sums_x, nullptr, true);
    return cudaGetLastError();
}

cudaError_t launch_validate(const DevGraph &g, int32_t num_labels, int *err, cudaStream_t st) {
    LAUNCHED(1);
    validate_kernel<<<blocks_for(g.n), kThreads, 0, st>>>(g, num_labels, err);
    return cudaGetLastError();
}

cudaError_t launch_prepare(const DevGraph &g, int64_t *piece_cnt, int32_t *end_off, int32_t *rank,
                           int32_t *cls_size, cudaStream_t st) {
    LAUNCHED(1);
    prepare_kernel<<<blocks_for(g.n), kThreads, 0, st>>>(g, piece_cnt, end_off, rank, cls_size);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ unit counts

namespace {
__global__ void unit_counts_kernel(const DevGraph g, const int32_t *fv, int64_t fN, int64_t e0, int64_t ne, int L,
                                   int V, int64_t quota, int64_t edge_quota, uint64_t qseed, int64_t *cnt) {
    const int64_t nu = ne * L;
    for (int64_t u = gtid(); u < nu; u += gstride()) {
        const int64_t e = e0 + u / L;
        const int p = (int)(u % L);
        const int32_t v = fv[(int64_t)p * fN + e];
        if (V == FSM_EXPLORE_SV) {   // single-vertex exploration: one candidate per neighbour of v
            cnt[u] = g.prow[v + 1] - g.prow[v];
            continue;
        }
        int64_t c = g.ppc[v];
        if (L == 2) {
            // centre pairs restricted to those with an end below the other vertex of s
            const int32_t w = fv[(int64_t)(1 - p) * fN + e];
            const int32_t rb = g.prow[v], d = g.prow[v + 1] - rb;
            const int32_t pos = count_below(g.pcol + rb, d, w);   // w's position in v's list
            c += centre_pairs(d, pos) - (int64_t)d * (d - 1) / 2;
            if (V == FSM_EXPLORE_TV_QUOTA && edge_quota > 0 && !quota_edge_kept(qseed, v, pos, d, edge_quota)) c = 0;
        }
        if (V == FSM_EXPLORE_TV_QUOTA && quota > 0 && c > quota) c = quota;
        cnt[u] = c;
    }
}

__global__ void fill_u64_kernel(unsigned long long *p, unsigned long long v, int64_t n) {
    for (int64_t i = gtid(); i < n; i += gstride()) p[i] = v;
}

__global__ void qp_compact_kernel(const unsigned long long *keys, int64_t cap, int64_t *slots,
                                  unsigned long long *n_out) {
    for (int64_t s = gtid(); s < cap; s += gstride()) {
        if (keys[s] != FSM_EMPTY_KEY) {
            const unsigned long long q = atomicAdd(n_out, 1ull);
            slots[q] = s;
        }
    }
}
} // namespace

cudaError_t launch_tri_words(const DevGraph &g, int32_t dmin, int64_t *words, cudaStream_t st) {
    LAUNCHED(1);
    tri_words_kernel<<<blocks_for(g.n), kThreads, 0, st>>>(g, dmin, words);
    return cudaGetLastError();
}

cudaError_t launch_tri_bits(const DevGraph &g, int32_t dmin, const int64_t *off, int64_t *tri_off, uint32_t *bits,
                            cudaStream_t st) {
    LAUNCHED(1);
    tri_bits_kernel<<<blocks_for(g.n * 32), kThreads, 0, st>>>(g, dmin, off, tri_off, bits);
    return cudaGetLastError();
}

cudaError_t launch_unit_counts(const DevGraph &g, const int32_t *fv, int64_t fN, int64_t e0, int64_t ne, int L,
                               int V, int64_t quota, int64_t edge_quota, uint64_t qseed, int64_t *cnt,
                               cudaStream_t st) {
    LAUNCHED(1);
    unit_counts_kernel<<<blocks_for(ne * L), kThreads, 0, st>>>(g, fv, fN, e0, ne, L, V, quota, edge_quota, qseed,
                                                                cnt);
    return cudaGetLastError();
}

namespace {
__global__ void unit_bytes_kernel(const int32_t *row_ptr, const int64_t *piece_cnt, const int32_t *fv, int64_t fN,
                                  int64_t e0, int64_t ne, int L, int V, unsigned long long *sum) {
    const int64_t nu = ne * L;
    unsigned long long s = 0;
    for (int64_t u = gtid(); u < nu; u += gstride()) {
        const int64_t e = e0 + u / L;
        const int32_t v = fv[(int64_t)(u % L) * fN + e];
        const int64_t d = row_ptr[v + 1] - row_ptr[v];
        // single-vertex exploration reads only the key vertex's list
        const int64_t ends = V == FSM_EXPLORE_SV ? 0 : piece_cnt[v] - d * (d - 1) / 2;
        s += 4ull * (unsigned long long)(d + ends);
        if (u % L == 0) s += 4ull * (unsigned long long)(L + 1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(sum, s);
}
} // namespace

cudaError_t launch_unit_bytes(const int32_t *row_ptr, const int64_t *piece_cnt, const int32_t *fv, int64_t fN,
                              int64_t e0, int64_t ne, int L, int V, unsigned long long *sum, cudaStream_t st) {
    LAUNCHED(1);
    unit_bytes_kernel<<<blocks_for(ne * L), kThreads, 0, st>>>(row_ptr, piece_cnt, fv, fN, e0, ne, L, V, sum);
    return cudaGetLastError();
}

namespace {
__global__ void group_kernel(const int32_t *fv, const int32_t *fpid, int64_t N, int L, const int64_t *off,
                             unsigned long long *cursor, int32_t *out_v, int32_t *out_pid) {
    for (int64_t e = gtid(); e < N; e += gstride()) {
        const int32_t p = fpid[e];
        const int64_t pos = off[p] + (int64_t)atomicAdd(cursor + p, 1ull);
        for (int c = 0; c < L; ++c) out_v[(int64_t)c * N + pos] = fv[(int64_t)c * N + e];
        out_pid[pos] = p;
    }
}
__global__ void u64_to_i64_kernel(const unsigned long long *in, int64_t *out, int64_t n) {
    for (int64_t i = gtid(); i < n; i += gstride()) out[i] = (int64_t)in[i];
}
} // namespace

cudaError_t launch_group_by_pattern(const int32_t *fv, const int32_t *fpid, int64_t N, int L, const int64_t *off,
                                    unsigned long long *cursor, int32_t *out_v, int32_t *out_pid, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    LAUNCHED(1);
    group_kernel<<<blocks_for(N), kThreads, 0, st>>>(fv, fpid, N, L, off, cursor, out_v, out_pid);
    return cudaGetLastError();
}

cudaError_t launch_u64_to_i64(const unsigned long long *in, int64_t *out, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    LAUNCHED(1);
    u64_to_i64_kernel<<<blocks_for(n), kThreads, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_fill_u64(unsigned long long *p, unsigned long long v, int64_t n, cudaStream_t st) {
    LAUNCHED(1);
    fill_u64_kernel<<<blocks_for(n), kThreads, 0, st>>>(p, v, n);
    return cudaGetLastError();
}

cudaError_t launch_qp_compact(const unsigned long long *keys, int64_t cap, int64_t *slots,
                              unsigned long long *n_out, cudaStream_t st) {
    LAUNCHED(1);
    qp_compact_kernel<<<blocks_for(cap), kThreads, 0, st>>>(keys, cap, slots, n_out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ canonical codes

namespace {

__global__ void qp_canon_kernel(int L, int V, const unsigned long long *keys, const int64_t *slots, int64_t nq,
                                const uint64_t *pat_lab8, const uint64_t *pat_adj8, CodeRec *recs,
                                uint64_t *perm_out) {
    for (int64_t q = gtid(); q < nq; q += gstride()) {
        const int64_t slot = slots[q];
        int K, labH[FSM_MAXK];
        uint32_t adjH[FSM_MAXK];
        key_graph(V, L, keys[slot], pat_lab8, pat_adj8, K, labH, adjH);
        unsigned long long cl;
        uint64_t ca, inv;
        canonicalise(K, labH, adjH, cl, ca, inv);
        recs[q].lab = cl;
        recs[q].adj = ca;
        recs[q].idx = (uint32_t)q;
        perm_out[slot] = inv;
    }
}

__device__ __forceinline__ bool rec_less(const CodeRec &a, const CodeRec &b) {
    if (a.lab != b.lab) return a.lab < b.lab;
    if (a.adj != b.adj) return a.adj < b.adj;
    return a.idx < b.idx;
}

__global__ void bitonic_step_kernel(CodeRec *r, int64_t M, int64_t j, int64_t k) {
    for (int64_t t = gtid(); t < M; t += gstride()) {
        const int64_t p = t ^ j;
        if (p <= t) continue;
        const bool up = (t & k) == 0;
        CodeRec a = r[t], b = r[p];
        if (up ? rec_less(b, a) : rec_less(a, b)) { r[t] = b; r[p] = a; }
    }
}

__global__ void pad_recs_kernel(CodeRec *r, int64_t n, int64_t M) {
    for (int64_t t = n + gtid(); t < M; t += gstride()) {
        r[t].lab = ~0ull; r[t].adj = ~0ull; r[t].idx = ~0u;
    }
}

__global__ void boundary_flags_kernel(const CodeRec *r, int64_t n, int64_t *flag) {
    for (int64_t t = gtid(); t < n; t += gstride())
        flag[t] = (t == 0 || r[t].lab != r[t - 1].lab || r[t].adj != r[t - 1].adj) ? 1 : 0;
}

__global__ void assign_kernel(const CodeRec *r, int64_t n, const int64_t *slots, const int64_t *flag,
                              const int64_t *ids, int32_t *qp_pattern, unsigned long long *pat_lab,
                              uint64_t *pat_adj) {
    for (int64_t t = gtid(); t < n; t += gstride()) {
        const int64_t pid = ids[t] + flag[t] - 1;
        qp_pattern[slots[r[t].idx]] = (int32_t)pid;
        if (flag[t]) { pat_lab[pid] = r[t].lab; pat_adj[pid] = r[t].adj; }
    }
}

__global__ void orbits_kernel(int K, const unsigned long long *pat_lab, const uint64_t *pat_adj, int64_t np,
                              uint64_t *orbit, int32_t *min_orbit) {
    for (int64_t P = gtid(); P < np; P += gstride()) {
        int rep[FSM_MAXK];
        orbit_reps(K, pat_lab[P], pat_adj[P], rep);
        uint64_t o = 0;
        int mn = K;
        for (int c = 0; c < K; ++c) {
            o |= nib_put(c, rep[c]);
            if (rep[c] == c) {
                int sz = 0;
                for (int x = 0; x < K; ++x) sz += rep[x] == c;
                if (sz < mn) mn = sz;
            }
        }
        orbit[P] = o;
        min_orbit[P] = mn;
    }
}

__global__ void pattern_counts_kernel(const int64_t *slots, int64_t nq, const int32_t *qp_pattern,
                                      const unsigned long long *qp_count, unsigned long long *pat_count) {
    for (int64_t q = gtid(); q < nq; q += gstride()) {
        const int64_t s = slots[q];
        atomicAdd(pat_count + qp_pattern[s], qp_count[s]);
    }
}

__global__ void domain_sizes_kernel(int K, const unsigned long long *pat_lab, const uint64_t *orbit,
                                    const int32_t *min_orbit, const unsigned long long *pat_count, int64_t np,
                                    int64_t t, const int32_t *cls_size, uint8_t *live, int64_t *words) {
    for (int64_t P = gtid(); P < np; P += gstride()) {
        const bool lv = (unsigned long long)min_orbit[P] * pat_count[P] >= (unsigned long long)t;
        live[P] = lv ? 1 : 0;
        for (int c = 0; c < FSM_MAXK; ++c) {
            int64_t w = 0;
            if (lv && c < K && nib_get(orbit[P], c) == c) w = ((int64_t)cls_size[clab_get(pat_lab[P], c)] + 31) / 32;
            words[P * FSM_MAXK + c] = w;
        }
    }
}

__global__ void domain_offsets_kernel(const int64_t *words, const int64_t *scanned, int64_t n8, int64_t *off) {
    for (int64_t x = gtid(); x < n8; x += gstride()) off[x] = words[x] > 0 ? scanned[x] : -1;
}

// one warp per (pattern, orbit representative)
__global__ void support_kernel(int K, const uint64_t *orbit, const uint8_t *live, const int64_t *dom_off,
                               const int64_t *words, const uint32_t *dom, int64_t np,
                               unsigned long long *sigma) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = np * FSM_MAXK;
    for (int64_t w = gtid() >> 5; w < nw; w += gstride() >> 5) {
        const int64_t P = w / FSM_MAXK;
        const int c = (int)(w % FSM_MAXK);
        if (!live[P] || c >= K || nib_get(orbit[P], c) != c) continue;
        const uint32_t *b = dom + dom_off[w];
        const int64_t n = words[w];
        unsigned long long s = 0;
        for (int64_t x = lane; x < n; x += 32) s += __popc(b[x]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) atomicMin(sigma + P, s);
    }
}

__global__ void freq_flags_kernel(const unsigned long long *sigma, int64_t np, int64_t t, int64_t *flag) {
    for (int64_t P = gtid(); P < np; P += gstride())
        flag[P] = (sigma[P] != ~0ull && sigma[P] >= (unsigned long long)t) ? 1 : 0;
}

__global__ void new_ids_kernel(const int64_t *flag, const int64_t *scanned, int64_t np, int32_t *newid) {
    for (int64_t P = gtid(); P < np; P += gstride()) newid[P] = flag[P] ? (int32_t)scanned[P] : -1;
}

__global__ void gather_frequent_kernel(int K, const int32_t *newid, int64_t np, const unsigned long long *pat_lab,
                                       const uint64_t *pat_adj, const unsigned long long *sigma,
                                       const unsigned long long *pat_count, unsigned long long *o_lab,
                                       uint64_t *o_adj, unsigned long long *o_sigma, unsigned long long *o_count,
                                       uint64_t *o_lab8, uint64_t *o_adj8) {
    for (int64_t P = gtid(); P < np; P += gstride()) {
        const int32_t id = newid[P];
        if (id < 0) continue;
        o_lab[id] = pat_lab[P];
        o_adj[id] = pat_adj[P];
        o_sigma[id] = sigma[P];
        o_count[id] = pat_count[P];
        if (o_lab8 && K <= 8) {
            int lab[FSM_MAXK];
            uint32_t adj[FSM_MAXK];
            decode_code(K, pat_lab[P], pat_adj[P], lab, adj);
            uint64_t l8 = 0, a8 = 0;
            for (int c = 0; c < K; ++c) {
                l8 |= (uint64_t)(lab[c] & 0xff) << (8 * c);
                a8 |= (uint64_t)(adj[c] & 0xff) << (8 * c);
            }
            o_lab8[id] = l8;
            o_adj8[id] = a8;
        }
    }
}

__global__ void sum_frequent_kernel(const int32_t *newid, const unsigned long long *pat_count, int64_t np,
                                    unsigned long long *sum) {
    unsigned long long s = 0;
    for (int64_t P = gtid(); P < np; P += gstride())
        if (newid[P] >= 0) s += pat_count[P];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(sum, s);
}

} // namespace

cudaError_t launch_qp_canon(int L, int V, const unsigned long long *keys, const int64_t *slots, int64_t nq,
                            const uint64_t *pat_lab8, const uint64_t *pat_adj8, CodeRec *recs,
                            uint64_t *perm, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    LAUNCHED(1);
    qp_canon_kernel<<<blocks_for(nq, 128), 128, 0, st>>>(L, V, keys, slots, nq, pat_lab8, pat_adj8, recs, perm);
    return cudaGetLastError();
}

cudaError_t launch_sort_codes(CodeRec *recs, int64_t n, cudaStream_t st) {
    if (n <= 1) return cudaSuccess;
    int64_t M = 1;
    while (M < n) M <<= 1;
    LAUNCHED(1);
    pad_recs_kernel<<<blocks_for(M - n + 1), kThreads, 0, st>>>(recs, n, M);
    for (int64_t k = 2; k <= M; k <<= 1)
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            LAUNCHED(1);
            bitonic_step_kernel<<<blocks_for(M), kThreads, 0, st>>>(recs, M, j, k);
        }
    return cudaGetLastError();
}

cudaError_t launch_assign_patterns(const CodeRec *recs, int64_t n, const int64_t *slots, int64_t *flag,
                                   int64_t *ids, void *scan_tmp, int32_t *qp_pattern,
                                   unsigned long long *pat_lab, uint64_t *pat_adj, cudaStream_t st) {
    if (n <= 0) return cudaMemsetAsync(ids, 0, sizeof(int64_t), st);
    LAUNCHED(1);
    boundary_flags_kernel<<<blocks_for(n), kThreads, 0, st>>>(recs, n, flag);
    cudaError_t e = launch_scan_i64(flag, ids, n, scan_tmp, st);
    if (e != cudaSuccess) return e;
    LAUNCHED(1);
    assign_kernel<<<blocks_for(n), kThreads, 0, st>>>(recs, n, slots, flag, ids, qp_pattern, pat_lab, pat_adj);
    return cudaGetLastError();
}

cudaError_t launch_orbits(int K, const unsigned long long *pat_lab, const uint64_t *pat_adj, int64_t np,
                          uint64_t *orbit, int32_t *min_orbit, cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    LAUNCHED(1);
    orbits_kernel<<<blocks_for(np, 128), 128, 0, st>>>(K, pat_lab, pat_adj, np, orbit, min_orbit);
    return cudaGetLastError();
}

cudaError_t launch_pattern_counts(const int64_t *slots, int64_t nq, const int32_t *qp_pattern,
                                  const unsigned long long *qp_count, unsigned long long *pat_count,
                                  cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    LAUNCHED(1);
    pattern_counts_kernel<<<blocks_for(nq), kThreads, 0, st>>>(slots, nq, qp_pattern, qp_count, pat_count);
    return cudaGetLastError();
}

cudaError_t launch_domain_sizes(int K, const unsigned long long *pat_lab, const uint64_t *orbit,
                                const int32_t *min_orbit, const unsigned long long *pat_count,
                                int64_t np, int64_t t, const int32_t *cls_size, uint8_t *live,
                                int64_t *words, cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    LAUNCHED(1);
    domain_sizes_kernel<<<blocks_for(np), kThreads, 0, st>>>(K, pat_lab, orbit, min_orbit, pat_count, np, t,
                                                           cls_size, live, words);
    return cudaGetLastError();
}

cudaError_t launch_domain_offsets(const int64_t *words, const int64_t *scanned, int64_t n8, int64_t *off,
                                  cudaStream_t st) {
    if (n8 <= 0) return cudaSuccess;
    LAUNCHED(1);
    domain_offsets_kernel<<<blocks_for(n8), kThreads, 0, st>>>(words, scanned, n8, off);
    return cudaGetLastError();
}

cudaError_t launch_support(int K, const uint64_t *orbit, const uint8_t *live, const int64_t *dom_off,
                           const int64_t *words, const uint32_t *dom, int64_t np,
                           unsigned long long *sigma, cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    LAUNCHED(1);
    support_kernel<<<blocks_for(np * FSM_MAXK * 32), kThreads, 0, st>>>(K, orbit, live, dom_off, words, dom, np, sigma);
    return cudaGetLastError();
}

cudaError_t launch_freq_flags(const unsigned long long *sigma, int64_t np, int64_t t, int64_t *flag,
                              cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    LAUNCHED(1);
    freq_flags_kernel<<<blocks_for(np), kThreads, 0, st>>>(sigma, np, t, flag);
    return cudaGetLastError();
}

cudaError_t launch_new_ids(const int64_t *flag, const int64_t *scanned, int64_t np, int32_t *newid,
                           cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    LAUNCHED(1);
    new_ids_kernel<<<blocks_for(np), kThreads, 0, st>>>(flag, scanned, np, newid);
    return cudaGetLastError();
}

cudaError_t launch_gather_frequent(int K, const int32_t *newid, int64_t np, const unsigned long long *pat_lab,
                                   const uint64_t *pat_adj, const unsigned long long *sigma,
                                   const unsigned long long *pat_count, unsigned long long *o_lab,
                                   uint64_t *o_adj, unsigned long long *o_sigma, unsigned long long *o_count,
                                   uint64_t *o_lab8, uint64_t *o_adj8, cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    LAUNCHED(1);
    gather_frequent_kernel<<<blocks_for(np), kThreads, 0, st>>>(K, newid, np, pat_lab, pat_adj, sigma, pat_count,
                                                              o_lab, o_adj, o_sigma, o_count, o_lab8, o_adj8);
    return cudaGetLastError();
}

cudaError_t launch_sum_frequent(const int32_t *newid, const unsigned long long *pat_count, int64_t np,
                                unsigned long long *sum, cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    LAUNCHED(1);
    sum_frequent_kernel<<<blocks_for(np), kThreads, 0, st>>>(newid, pat_count, np, sum);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ base levels

namespace {

__global__ void level1_flags_kernel(const DevGraph g, const int32_t *label_newid, int64_t *flag) {
    for (int64_t v = gtid(); v < g.n; v += gstride()) flag[v] = label_newid[g.labels[v]] >= 0 ? 1 : 0;
}

__global__ void level1_write_kernel(const DevGraph g, const int32_t *label_newid, const int64_t *flag,
                                    const int64_t *scanned, int32_t *fv, int32_t *fpid) {
    for (int64_t v = gtid(); v < g.n; v += gstride()) {
        if (!flag[v]) continue;
        const int64_t pos = scanned[v];
        fv[pos] = (int32_t)v;
        fpid[pos] = label_newid[g.labels[v]];
    }
}

__global__ void level2_offsets_kernel(int32_t NL, const int32_t *cls_size, int64_t *pair_off, int64_t *total) {
    if (gtid() != 0) return;
    int64_t run = 0;
    for (int lo = 0; lo < NL; ++lo)
        for (int hi = 0; hi < NL; ++hi) {
            const int64_t x = ((int64_t)lo * NL + hi) * 2;
            if (hi < lo) { pair_off[x] = -1; pair_off[x + 1] = -1; continue; }
            pair_off[x] = run;
            run += ((int64_t)cls_size[lo] + 31) / 32;
            if (hi > lo) { pair_off[x + 1] = run; run += ((int64_t)cls_size[hi] + 31) / 32; }
            else pair_off[x + 1] = -1;
        }
    *total = run;
}

__device__ __forceinline__ void set_bit(uint32_t *dom, int64_t off, int32_t r) {
    uint32_t *w = dom + off + (r >> 5);
    const uint32_t bit = 1u << (r & 31);
    if (!(__ldcg(w) & bit)) atomicOr(w, bit);
}

__global__ void level2_domains_kernel(const DevGraph g, int32_t NL, const int64_t *pair_off, uint32_t *dom,
                                      unsigned long long *pair_count) {
    for (int64_t u = gtid(); u < g.n; u += gstride()) {
        const int lu = g.labels[u];
        const int32_t ru = g.rank[u];
        for (int32_t j = g.row_ptr[u]; j < g.row_ptr[u + 1]; ++j) {
            const int32_t w = g.col[j];
            if (w < u) continue;
            const int lw = g.labels[w];
            const int lo = lu < lw ? lu : lw, hi = lu < lw ? lw : lu;
            const int64_t x = ((int64_t)lo * NL + hi) * 2;
            atomicAdd(pair_count + (x >> 1), 1ull);
            if (lo == hi) {
                set_bit(dom, pair_off[x], ru);
                set_bit(dom, pair_off[x], g.rank[w]);
            } else if (lu < lw) {
                set_bit(dom, pair_off[x], ru);
                set_bit(dom, pair_off[x + 1], g.rank[w]);
            } else {
                set_bit(dom, pair_off[x], g.rank[w]);
                set_bit(dom, pair_off[x + 1], ru);
            }
        }
    }
}

// one warp per label pair (lo <= hi)
__global__ void level2_support_kernel(int32_t NL, const int32_t *cls_size, const int64_t *pair_off,
                                      const uint32_t *dom, unsigned long long *sigma) {
    const int lane = threadIdx.x & 31;
    const int64_t np = (int64_t)NL * NL;
    for (int64_t w = gtid() >> 5; w < np; w += gstride() >> 5) {
        const int lo = (int)(w / NL), hi = (int)(w % NL);
        if (hi < lo) { if (lane == 0) sigma[w] = 0; continue; }
        unsigned long long s0 = 0, s1 = 0;
        const int64_t n0 = ((int64_t)cls_size[lo] + 31) / 32;
        for (int64_t x = lane; x < n0; x += 32) s0 += __popc(dom[pair_off[w * 2] + x]);
        if (hi > lo) {
            const int64_t n1 = ((int64_t)cls_size[hi] + 31) / 32;
            for (int64_t x = lane; x < n1; x += 32) s1 += __popc(dom[pair_off[w * 2 + 1] + x]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        if (lane == 0) sigma[w] = (hi > lo) ? (s0 < s1 ? s0 : s1) : s0;
    }
}

__global__ void level2_flags_kernel(const DevGraph g, int32_t NL, const int32_t *pair_newid, int64_t *flag) {
    for (int64_t u = gtid(); u < g.n; u += gstride()) {
        const int lu = g.labels[u];
        int64_t c = 0;
        for (int32_t j = g.row_ptr[u]; j < g.row_ptr[u + 1]; ++j) {
            const int32_t w = g.col[j];
            if (w < u) continue;
            const int lw = g.labels[w];
            const int lo = lu < lw ? lu : lw, hi = lu < lw ? lw : lu;
            c += pair_newid[lo * NL + hi] >= 0;
        }
        flag[u] = c;
    }
}

__global__ void level2_write_kernel(const DevGraph g, int32_t NL, const int32_t *pair_newid,
                                    const int64_t *scanned, int32_t *fv, int64_t fN, int32_t *fpid) {
    for (int64_t u = gtid(); u < g.n; u += gstride()) {
        const int lu = g.labels[u];
        int64_t pos = scanned[u];
        for (int32_t j = g.row_ptr[u]; j < g.row_ptr[u + 1]; ++j) {
            const int32_t w = g.col[j];
            if (w < u) continue;
            const int lw = g.labels[w];
            const int lo = lu < lw ? lu : lw, hi = lu < lw ? lw : lu;
            const int32_t id = pair_newid[lo * NL + hi];
            if (id < 0) continue;
            // canonical order: smaller label first; equal labels: smaller id first (u < w)
            const bool u_first = lu <= lw;
            fv[pos] = u_first ? (int32_t)u : w;
            fv[fN + pos] = u_first ? w : (int32_t)u;
            fpid[pos] = id;
            ++pos;
        }
    }
}

__global__ void piece_table_kernel(const unsigned long long *lab, const uint64_t *adj, int64_t n, uint8_t *pf) {
    for (int64_t P = gtid(); P < n; P += gstride()) {
        const int l0 = clab_get(lab[P], 0), l1 = clab_get(lab[P], 1), l2 = clab_get(lab[P], 2);
        const uint32_t a01 = (adj[P] >> 2) & 1u, a02 = (adj[P] >> 1) & 1u, a12 = adj[P] & 1u;
        uint32_t idx;
        if (a01 && a02 && a12) idx = tri_index(l0, l1, l2);
        else if (a01 && a02) idx = wedge_index(l0, l1, l2);
        else if (a01 && a12) idx = wedge_index(l1, l0, l2);
        else idx = wedge_index(l2, l0, l1);
        pf[idx] = 1;
    }
}

} // namespace

cudaError_t launch_level1_frontier(const DevGraph &g, const int32_t *label_newid, int64_t *flag,
                                   int64_t *scanned, void *scan_tmp, int32_t *fv, int32_t *fpid,
                                   cudaStream_t st) {
    LAUNCHED(1);
    level1_flags_kernel<<<blocks_for(g.n), kThreads, 0, st>>>(g, label_newid, flag);
    cudaError_t e = launch_scan_i64(flag, scanned, g.n, scan_tmp, st);
    if (e != cudaSuccess) return e;
    LAUNCHED(1);
    level1_write_kernel<<<blocks_for(g.n), kThreads, 0, st>>>(g, label_newid, flag, scanned, fv, fpid);
    return cudaGetLastError();
}

cudaError_t launch_level2_offsets(int32_t NL, const int32_t *cls_size, int64_t *pair_off,
                                  int64_t *total_words, cudaStream_t st) {
    LAUNCHED(1);
    level2_offsets_kernel<<<1, 32, 0, st>>>(NL, cls_size, pair_off, total_words);
    return cudaGetLastError();
}

cudaError_t launch_level2_domains(const DevGraph &g, int32_t NL, const int64_t *pair_off,
                                  uint32_t *dom, unsigned long long *pair_count, cudaStream_t st) {
    LAUNCHED(1);
    level2_domains_kernel<<<blocks_for(g.n), kThreads, 0, st>>>(g, NL, pair_off, dom, pair_count);
    return cudaGetLastError();
}

cudaError_t launch_level2_support(int32_t NL, const int32_t *cls_size, const int64_t *pair_off,
                                  const uint32_t *dom, unsigned long long *sigma, cudaStream_t st) {
    LAUNCHED(1);
    level2_support_kernel<<<blocks_for((int64_t)NL * NL * 32), kThreads, 0, st>>>(NL, cls_size, pair_off, dom, sigma);
    return cudaGetLastError();
}

cudaError_t launch_level2_frontier(const DevGraph &g, int32_t NL, const int32_t *pair_newid,
                                   int64_t *flag, int64_t *scanned, void *scan_tmp, int32_t *fv,
                                   int64_t fN, int32_t *fpid, cudaStream_t st) {
    LAUNCHED(1);
    level2_flags_kernel<<<blocks_for(g.n), kThreads, 0, st>>>(g, NL, pair_newid, flag);
    cudaError_t e = launch_scan_i64(flag, scanned, g.n, scan_tmp, st);
    if (e != cudaSuccess) return e;
    LAUNCHED(1);
    level2_write_kernel<<<blocks_for(g.n), kThreads, 0, st>>>(g, NL, pair_newid, scanned, fv, fN, fpid);
    return cudaGetLastError();
}

namespace {
__global__ void level1_tables_kernel(int32_t NL, const int32_t *cls_size, int64_t t, int32_t *label_newid,
                                     uint64_t *lab8, uint64_t *adj8, unsigned long long *clab, uint64_t *cadj,
                                     unsigned long long *sigma, unsigned long long *count,
                                     unsigned long long *n_freq) {
    if (gtid() != 0) return;
    int32_t id = 0;
    for (int l = 0; l < NL; ++l) {
        // size-1 pattern of label l: every vertex of the class is an image (Definition 2)
        const int64_t s = cls_size[l];
        if (s >= t && s > 0) {
            label_newid[l] = id;
            lab8[id] = (uint64_t)l;
            adj8[id] = 0;
            clab[id] = clab_put(0, l);
            cadj[id] = 0;
            sigma[id] = (unsigned long long)s;
            count[id] = (unsigned long long)s;
            ++id;
        } else {
            label_newid[l] = -1;
        }
    }
    *n_freq = (unsigned long long)id;
}

__global__ void level2_tables_kernel(int32_t NL, const unsigned long long *pair_sigma,
                                     const unsigned long long *pair_count, int64_t t, int32_t *pair_newid,
                                     uint64_t *lab8, uint64_t *adj8, unsigned long long *clab, uint64_t *cadj,
                                     unsigned long long *sigma, unsigned long long *count,
                                     unsigned long long *n_freq) {
    if (gtid() != 0) return;
    int32_t id = 0;
    for (int lo = 0; lo < NL; ++lo)
        for (int hi = 0; hi < NL; ++hi) {
            const int64_t x = (int64_t)lo * NL + hi;
            if (hi >= lo && pair_count[x] > 0 && pair_sigma[x] >= (unsigned long long)t) {
                pair_newid[x] = id;
                lab8[id] = (uint64_t)lo | ((uint64_t)hi << 8);
                adj8[id] = 0x0102ull;                  // row 0 = {1}, row 1 = {0}
                clab[id] = clab_put(0, lo) | clab_put(1, hi);
                cadj[id] = 1ull;
                sigma[id] = pair_sigma[x];
                count[id] = pair_count[x];
                ++id;
            } else {
                pair_newid[x] = -1;
            }
        }
    *n_freq = (unsigned long long)id;
}
} // namespace

cudaError_t launch_level1_tables(int32_t NL, const int32_t *cls_size, int64_t t, int32_t *label_newid,
                                 uint64_t *lab8, uint64_t *adj8, unsigned long long *clab, uint64_t *cadj,
                                 unsigned long long *sigma, unsigned long long *count,
                                 unsigned long long *n_freq, cudaStream_t st) {
    LAUNCHED(1);
    level1_tables_kernel<<<1, 32, 0, st>>>(NL, cls_size, t, label_newid, lab8, adj8, clab, cadj, sigma, count, n_freq);
    return cudaGetLastError();
}

cudaError_t launch_level2_tables(int32_t NL, const unsigned long long *pair_sigma,
                                 const unsigned long long *pair_count, int64_t t, int32_t *pair_newid,
                                 uint64_t *lab8, uint64_t *adj8, unsigned long long *clab, uint64_t *cadj,
                                 unsigned long long *sigma, unsigned long long *count,
                                 unsigned long long *n_freq, cudaStream_t st) {
    LAUNCHED(1);
    level2_tables_kernel<<<1, 32, 0, st>>>(NL, pair_sigma, pair_count, t, pair_newid, lab8, adj8, clab, cadj,
                                           sigma, count, n_freq);
    return cudaGetLastError();
}

namespace {

__global__ void class_offsets_kernel(int32_t NL, const int32_t *cls_size, int64_t *cls_off) {
    if (gtid() != 0) return;
    int64_t run = 0;
    for (int l = 0; l < NL; ++l) { cls_off[l] = run; run += cls_size[l]; }
    cls_off[NL] = run;
}

__global__ void by_rank_kernel(const DevGraph g, const int64_t *cls_off, int32_t *by_rank) {
    for (int64_t v = gtid(); v < g.n; v += gstride()) by_rank[cls_off[g.labels[v]] + g.rank[v]] = (int32_t)v;
}

// one warp per (pattern, canonical position): popcount and mean log1p(degree) of the orbit's
// sampled domain; lane 0 of the position-0 warp also writes the scalars
// Features, per (pattern, canonical position) warp: the label frequency of the position and the
// mean log1p(degree) over the sampled domain of its orbit; the orbit's popcount goes to pop[].
__global__ void features_pos_kernel(int K, const unsigned long long *pat_lab, const uint64_t *orbit,
                                    const int64_t *dom_off, const int64_t *words, const uint32_t *dom,
                                    const int32_t *cls_size, const int64_t *cls_off, const int32_t *by_rank,
                                    const int32_t *row_ptr, int32_t n, int64_t np, unsigned long long *pop,
                                    float *feat) {
    const int lane = threadIdx.x & 31;
    // sampled levels have K <= 8: eight feature slots per block
    const int64_t nw = np * 8;
    for (int64_t w = gtid() >> 5; w < nw; w += gstride() >> 5) {
        const int64_t P = w >> 3;
        const int c = (int)(w & 7);
        float *f = feat + P * 32;
        if (c >= K) {
            if (lane == 0) { f[8 + c] = 0.f; f[16 + c] = 0.f; pop[w] = 0; }
            continue;
        }
        const int o = nib_get(orbit[P], c);
        const int lab = clab_get(pat_lab[P], c);
        const int64_t off = dom_off[P * FSM_MAXK + o], nwd = words[P * FSM_MAXK + o];
        float sdeg = 0.f;
        unsigned long long cnt = 0;
        for (int64_t x = lane; x < nwd; x += 32) {
            uint32_t bits = dom[off + x];
            cnt += __popc(bits);
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const int32_t v = by_rank[cls_off[lab] + x * 32 + b];
                sdeg += log1pf((float)(row_ptr[v + 1] - row_ptr[v]));
            }
        }
#pragma unroll
        for (int s2 = 16; s2 > 0; s2 >>= 1) {
            sdeg += __shfl_xor_sync(0xffffffffu, sdeg, s2);
            cnt += __shfl_xor_sync(0xffffffffu, cnt, s2);
        }
        if (lane != 0) continue;
        f[8 + c] = logf((float)cls_size[lab] / (float)n);
        f[16 + c] = cnt ? sdeg / (float)cnt : 0.f;
        pop[w] = cnt;
    }
}

// Features, per pattern: the orbits' popcounts ascending (from pop[] at each orbit's
// representative) and the pattern-level entries.
__global__ void features_pat_kernel(int K, const uint64_t *pat_adj, const uint64_t *orbit,
                                    const unsigned long long *pat_count, int32_t n, float logp, float p, int64_t t,
                                    int64_t np, const int64_t *aut, const unsigned long long *pop, float *feat) {
    for (int64_t P = gtid(); P < np; P += gstride()) {
        float *f = feat + P * 32;
        float pc[8];
        int m = 0;
        unsigned long long mn = ~0ull;
        for (int c = 0; c < K; ++c) {
            if (nib_get(orbit[P], c) != c) continue;
            const unsigned long long q = pop[P * 8 + c];
            if (q < mn) mn = q;
            pc[m++] = log1pf((float)q);
        }
        for (int a = 1; a < m; ++a)
            for (int b = a; b > 0 && pc[b - 1] > pc[b]; --b) { float tt = pc[b]; pc[b] = pc[b - 1]; pc[b - 1] = tt; }
        for (int a = 0; a < 8; ++a) f[a] = a < m ? pc[a] : 0.f;
        f[24] = (float)K;
        f[25] = (float)__popcll(pat_adj[P]);
        f[26] = logp;
        f[27] = log1pf((float)pat_count[P]);
        f[28] = logf((float)t / (float)n);
        f[29] = logf((float)aut[P]);
        f[30] = logf(((float)mn + 1.f) / p);
        f[31] = logf((float)n);
    }
}

__global__ void aut_size_kernel(int K, const unsigned long long *pat_lab, const uint64_t *pat_adj, int64_t np,
                                int64_t *aut) {
    for (int64_t P = gtid(); P < np; P += gstride()) {
        int lab[FSM_MAXK], perm[FSM_MAXK], seg[FSM_MAXK];
        uint32_t adj[FSM_MAXK];
        decode_code(K, pat_lab[P], pat_adj[P], lab, adj);
        for (int c = 0; c < K; ++c) {
            perm[c] = c;
            seg[c] = (c > 0 && lab[c] == lab[c - 1]) ? seg[c - 1] : c;
        }
        int64_t a = 0;
        do {
            a += adj_code(K, adj, perm) == pat_adj[P];
        } while (next_label_perm(K, seg, perm));
        aut[P] = a;
    }
}

} // namespace

namespace {
__global__ void sample_count_kernel(const DevGraph g, uint64_t seed, uint64_t thr, int64_t *cnt) {
    for (int64_t v = gtid(); v < g.n; v += gstride()) {
        int64_t c = 0;
        for (int32_t j = g.row_ptr[v]; j < g.row_ptr[v + 1]; ++j) c += keep_edge(seed, thr, (int32_t)v, g.col[j]);
        cnt[v] = c;
    }
}
__global__ void sample_fill_kernel(const DevGraph g, uint64_t seed, uint64_t thr, const int64_t *prow64, int32_t *prow,
                                   int32_t *pcol) {
    for (int64_t v = gtid(); v < g.n; v += gstride()) {
        int64_t o = prow64[v];
        prow[v] = (int32_t)o;
        if (v == g.n - 1) prow[g.n] = (int32_t)prow64[g.n];
        for (int32_t j = g.row_ptr[v]; j < g.row_ptr[v + 1]; ++j)
            if (keep_edge(seed, thr, (int32_t)v, g.col[j])) pcol[o++] = g.col[j];
    }
}
__global__ void sample_pieces_kernel(int32_t n, const int32_t *prow, const int32_t *pcol, int32_t *pend, int64_t *ppc) {
    for (int64_t v = gtid(); v < n; v += gstride()) {
        const int64_t d = prow[v + 1] - prow[v];
        int64_t run = 0;
        for (int32_t j = prow[v]; j < prow[v + 1]; ++j) {
            pend[j] = (int32_t)run;
            const int32_t a = pcol[j];
            run += prow[a + 1] - prow[a];
        }
        ppc[v] = d * (d - 1) / 2 + run;
    }
}
} // namespace

cudaError_t launch_sample_count(const DevGraph &g, uint64_t seed, uint64_t thr, int64_t *cnt, cudaStream_t st) {
    LAUNCHED(1);
    sample_count_kernel<<<blocks_for(g.n), kThreads, 0, st>>>(g, seed, thr, cnt);
    return cudaGetLastError();
}

cudaError_t launch_sample_lists(const DevGraph &g, uint64_t seed, uint64_t thr, const int64_t *prow64, int32_t *prow,
                                int32_t *pcol, int32_t *pend, int64_t *ppc, cudaStream_t st) {
    LAUNCHED(2);
    sample_fill_kernel<<<blocks_for(g.n), kThreads, 0, st>>>(g, seed, thr, prow64, prow, pcol);
    sample_pieces_kernel<<<blocks_for(g.n), kThreads, 0, st>>>(g.n, prow, pcol, pend, ppc);
    return cudaGetLastError();
}

cudaError_t launch_by_rank(const DevGraph &g, int32_t NL, const int32_t *cls_size, int64_t *cls_off,
                           int32_t *by_rank, cudaStream_t st) {
    LAUNCHED(2);
    class_offsets_kernel<<<1, 32, 0, st>>>(NL, cls_size, cls_off);
    by_rank_kernel<<<blocks_for(g.n), kThreads, 0, st>>>(g, cls_off, by_rank);
    return cudaGetLastError();
}

cudaError_t launch_aut_size(int K, const unsigned long long *pat_lab, const uint64_t *pat_adj, int64_t np,
                            int64_t *aut, cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    LAUNCHED(1);
    aut_size_kernel<<<blocks_for(np, 128), 128, 0, st>>>(K, pat_lab, pat_adj, np, aut);
    return cudaGetLastError();
}

cudaError_t launch_features(int K, const unsigned long long *pat_lab, const uint64_t *pat_adj, const uint64_t *orbit,
                            const int64_t *dom_off, const int64_t *words, const uint32_t *dom,
                            const unsigned long long *pat_count, const int32_t *cls_size, const int64_t *cls_off,
                            const int32_t *by_rank, const int32_t *row_ptr, int32_t n, double p, int64_t t,
                            int64_t np, const int64_t *aut, float *feat, cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    unsigned long long *pop = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&pop, sizeof(unsigned long long) * (size_t)np * 8, st);
    if (e != cudaSuccess) return e;
    LAUNCHED(2);
    features_pos_kernel<<<blocks_for(np * 8 * 32), kThreads, 0, st>>>(K, pat_lab, orbit, dom_off, words, dom, cls_size,
                                                                      cls_off, by_rank, row_ptr, n, np, pop, feat);
    features_pat_kernel<<<blocks_for(np), kThreads, 0, st>>>(K, pat_adj, orbit, pat_count, n, (float)log(p), (float)p,
                                                             t, np, aut, pop, feat);
    e = cudaGetLastError();
    cudaFreeAsync(pop, st);
    return e;
}

namespace {

__device__ bool mask_conn(uint32_t m, const uint32_t *adj, int K) { return mask_connected(m, adj, K); }

__global__ void needed_parts_kernel(int K, const unsigned long long *lab, const uint64_t *adj, const uint8_t *uncertain,
                                    int64_t np, const unsigned long long *s_lab, const uint64_t *s_adj, int64_t s_np,
                                    uint8_t *need_s, uint8_t *need_piece) {
    for (int64_t P = gtid(); P < np; P += gstride()) {
        if (!uncertain[P]) continue;
        int lb[FSM_MAXK];
        uint32_t ad[FSM_MAXK];
        decode_code(K, lab[P], adj[P], lb, ad);
        const uint32_t all = (1u << K) - 1u;
        for (uint32_t l = 0; l <= all; ++l) {
            if (popc32(l) != 3) continue;
            uint32_t la[FSM_MAXK];
            for (int h = 0; h < K; ++h) la[h] = ad[h] & l;
            if (!mask_conn(l, la, K)) continue;
            // the piece: shape and labels of P restricted to l
            int v3[3], c = 0;
            for (int h = 0; h < K; ++h) if (l >> h & 1u) v3[c++] = h;
            const uint32_t e01 = ad[v3[0]] >> v3[1] & 1u, e02 = ad[v3[0]] >> v3[2] & 1u, e12 = ad[v3[1]] >> v3[2] & 1u;
            uint32_t pidx;
            if (e01 && e02 && e12) pidx = tri_index(lb[v3[0]], lb[v3[1]], lb[v3[2]]);
            else if (e01 && e02) pidx = wedge_index(lb[v3[0]], lb[v3[1]], lb[v3[2]]);
            else if (e01 && e12) pidx = wedge_index(lb[v3[1]], lb[v3[0]], lb[v3[2]]);
            else pidx = wedge_index(lb[v3[2]], lb[v3[0]], lb[v3[1]]);
            for (int q = 0; q < 3; ++q) {
                const uint32_t r = (all & ~l) | (1u << v3[q]);
                uint32_t ra[FSM_MAXK];
                for (int h = 0; h < K; ++h) ra[h] = ad[h] & r;
                if (!mask_conn(r, ra, K)) continue;
                need_piece[pidx] = 1;
                // canonical code of the (K-2)-vertex part, then its id among the stored patterns
                int sl[FSM_MAXK], map[FSM_MAXK], m = 0;
                for (int h = 0; h < K; ++h) if (r >> h & 1u) { map[h] = m; sl[m++] = lb[h]; }
                uint32_t sa[FSM_MAXK] = {0};
                for (int h = 0; h < K; ++h) {
                    if (!(r >> h & 1u)) continue;
                    for (int h2 = 0; h2 < K; ++h2)
                        if ((r >> h2 & 1u) && (ad[h] >> h2 & 1u)) sa[map[h]] |= 1u << map[h2];
                }
                unsigned long long cl;
                uint64_t ca, inv;
                canonicalise(m, sl, sa, cl, ca, inv);
                int64_t lo = 0, hi = s_np;
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (s_lab[mid] < cl || (s_lab[mid] == cl && s_adj[mid] < ca)) lo = mid + 1; else hi = mid;
                }
                if (lo < s_np && s_lab[lo] == cl && s_adj[lo] == ca) need_s[lo] = 1;
            }
        }
    }
}

__global__ void flag_keep_kernel(const int32_t *fpid, int64_t N, const uint8_t *keep, int64_t *flag) {
    for (int64_t e = gtid(); e < N; e += gstride()) flag[e] = keep[fpid[e]] ? 1 : 0;
}

__global__ void compact_frontier_kernel(const int32_t *fv, const int32_t *fpid, int64_t N, int L, const int64_t *flag,
                                        const int64_t *scanned, int32_t *out_v, int64_t outN, int32_t *out_pid) {
    for (int64_t e = gtid(); e < N; e += gstride()) {
        if (!flag[e]) continue;
        const int64_t pos = scanned[e];
        for (int c = 0; c < L; ++c) out_v[(int64_t)c * outN + pos] = fv[(int64_t)c * N + e];
        out_pid[pos] = fpid[e];
    }
}

__global__ void and_u8_kernel(uint8_t *a, const uint8_t *b, int64_t n) {
    for (int64_t i = gtid(); i < n; i += gstride()) a[i] = a[i] & b[i];
}

} // namespace

cudaError_t launch_needed_parts(int K, const unsigned long long *lab, const uint64_t *adj, const uint8_t *uncertain,
                                int64_t np, const unsigned long long *s_lab, const uint64_t *s_adj, int64_t s_np,
                                uint8_t *need_s, uint8_t *need_piece, cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    LAUNCHED(1);
    needed_parts_kernel<<<blocks_for(np, 64), 64, 0, st>>>(K, lab, adj, uncertain, np, s_lab, s_adj, s_np, need_s, need_piece);
    return cudaGetLastError();
}

cudaError_t launch_flag_count(const int32_t *fpid, int64_t N, const uint8_t *keep, int64_t *flag, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    LAUNCHED(1);
    flag_keep_kernel<<<blocks_for(N), kThreads, 0, st>>>(fpid, N, keep, flag);
    return cudaGetLastError();
}

cudaError_t launch_compact_frontier(const int32_t *fv, const int32_t *fpid, int64_t N, int L, const uint8_t *keep,
                                    int64_t *flag, int64_t *scanned, void *scan_tmp, int32_t *out_v, int64_t outN,
                                    int32_t *out_pid, cudaStream_t st) {
    (void)keep;
    if (N <= 0) return cudaSuccess;
    LAUNCHED(1);
    compact_frontier_kernel<<<blocks_for(N), kThreads, 0, st>>>(fv, fpid, N, L, flag, scanned, out_v, outN, out_pid);
    (void)scan_tmp;
    return cudaGetLastError();
}

namespace {
__global__ void keep_counts_kernel(const unsigned long long *count, const uint8_t *keep, int64_t np, unsigned long long *out) {
    for (int64_t P = gtid(); P < np; P += gstride()) out[P] = keep[P] ? count[P] : 0ull;
}
} // namespace

cudaError_t launch_keep_counts(const unsigned long long *count, const uint8_t *keep, int64_t np, unsigned long long *out,
                               cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    LAUNCHED(1);
    keep_counts_kernel<<<blocks_for(np), kThreads, 0, st>>>(count, keep, np, out);
    return cudaGetLastError();
}

cudaError_t launch_and_u8(uint8_t *a, const uint8_t *b, int64_t n, cudaStream_t st) {
    LAUNCHED(1);
    and_u8_kernel<<<blocks_for(n), kThreads, 0, st>>>(a, b, n);
    return cudaGetLastError();
}

namespace {
__global__ void decide_kernel(const float *pred, int64_t np, float logt, float delta, uint8_t *keep, uint8_t *unc) {
    for (int64_t P = gtid(); P < np; P += gstride()) {
        const float d = pred[P] - logt;
        keep[P] = d >= delta ? 1 : 0;
        unc[P] = (d < delta && d >= -delta) ? 1 : 0;
    }
}
} // namespace

cudaError_t launch_decide(const float *pred, int64_t np, float logt, float delta, uint8_t *keep, uint8_t *uncertain,
                          cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    LAUNCHED(1);
    decide_kernel<<<blocks_for(np), kThreads, 0, st>>>(pred, np, logt, delta, keep, uncertain);
    return cudaGetLastError();
}

namespace {
// MNI support of each pattern from the one-pass last level's orbit bitmaps: the pattern's entry
// in the code table gives its bitmap block; orbit representatives (ascending canonical
// position) hold ceil(|V_label| / 32) words each, in that order.  One warp per pattern.
__global__ void fused_support_kernel(int K, const unsigned long long *plab, const uint64_t *padj, const uint64_t *orbit,
                                     int64_t np, const unsigned long long *ckeys, const unsigned long long *coff,
                                     uint64_t cmask, const int32_t *cls_size, const uint32_t *pool,
                                     unsigned long long *sigma) {
    const int lane = threadIdx.x & 31;
    for (int64_t P = gtid() >> 5; P < np; P += gstride() >> 5) {
        const uint64_t pk = pack_code(K, plab[P], padj[P]);
        uint64_t h = mix64(pk) & cmask;
        int64_t ci = -1;
        for (uint64_t probe = 0; probe <= cmask; ++probe) {
            const unsigned long long cur = ckeys[h];
            if (cur == pk) { ci = (int64_t)h; break; }
            if (cur == FSM_EMPTY_KEY) break;
            h = (h + 1) & cmask;
        }
        if (ci < 0 || coff[ci] == 0ull) {   // cannot happen: every key was resolved before use
            if (lane == 0) sigma[P] = 0;
            continue;
        }
        const uint64_t off = coff[ci] - 1ull;
        uint64_t pre = 0;
        unsigned long long mn = ~0ull;
        for (int c = 0; c < K; ++c) {
            if (nib_get(orbit[P], c) != c) continue;
            const uint64_t nw = ((uint64_t)cls_size[clab_get(plab[P], c)] + 31) / 32;
            unsigned long long cnt = 0;
            for (uint64_t x = lane; x < nw; x += 32) cnt += __popc(pool[off + pre + x]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            if (cnt < mn) mn = cnt;
            pre += nw;
        }
        if (lane == 0) sigma[P] = mn;
    }
}

} // namespace

cudaError_t launch_fused_support(int K, const unsigned long long *plab, const uint64_t *padj, const uint64_t *orbit,
                                 int64_t np, const unsigned long long *ckeys, const unsigned long long *coff,
                                 uint64_t cmask, const int32_t *cls_size, const uint32_t *pool, unsigned long long *sigma,
                                 cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    LAUNCHED(1);
    fused_support_kernel<<<blocks_for(np * 32), kThreads, 0, st>>>(K, plab, padj, orbit, np, ckeys, coff, cmask, cls_size,
                                                                   pool, sigma);
    return cudaGetLastError();
}

namespace {
__global__ void slot_bases_kernel(int K, const int64_t *slots, int64_t nq, const int32_t *qp_pattern,
                                  const uint64_t *qp_perm, const uint8_t *live, const uint64_t *orbit,
                                  const int64_t *dom_off, int64_t *slot_base) {
    for (int64_t q = gtid(); q < nq; q += gstride()) {
        const int64_t slot = slots[q];
        const int32_t P = qp_pattern[slot];
        for (int h = 0; h < FSM_MAXK; ++h) {
            int64_t b = -1;
            if (h < K && live[P]) b = dom_off[(int64_t)P * FSM_MAXK + nib_get(orbit[P], nib_get(qp_perm[slot], h))];
            slot_base[slot * FSM_MAXK + h] = b;
        }
    }
}
} // namespace

cudaError_t launch_slot_bases(int K, const int64_t *slots, int64_t nq, const int32_t *qp_pattern,
                              const uint64_t *qp_perm, const uint8_t *live, const uint64_t *orbit,
                              const int64_t *dom_off, int64_t *slot_base, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    LAUNCHED(1);
    slot_bases_kernel<<<blocks_for(nq), kThreads, 0, st>>>(K, slots, nq, qp_pattern, qp_perm, live, orbit, dom_off,
                                                           slot_base);
    return cudaGetLastError();
}

cudaError_t launch_piece_table(const unsigned long long *lab, const uint64_t *adj, int64_t n,
                               uint8_t *piece_freq, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    LAUNCHED(1);
    piece_table_kernel<<<blocks_for(n), kThreads, 0, st>>>(lab, adj, n, piece_freq);
    return cudaGetLastError();
}

} // namespace fsm

namespace fsm {
namespace {
__global__ void stamp_time_kernel(unsigned long long *out) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    *out = t;
}
} // namespace

cudaError_t launch_stamp_time(unsigned long long *out, cudaStream_t st) {
    LAUNCHED(1);
    stamp_time_kernel<<<1, 1, 0, st>>>(out);
    return cudaGetLastError();
}
} // namespace fsm
