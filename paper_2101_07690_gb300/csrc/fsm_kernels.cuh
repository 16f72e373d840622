// fsm_kernels.cuh -- host-callable launchers for every kernel outside the extension kernel.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "fsm_device.cuh"

namespace fsm {

// One pattern's canonical code: the label word and the adjacency word of fsm_device.cuh
// (integer order on (lab, adj) is the lexicographic order of the code).  idx carries a payload
// through sorting.
struct CodeRec {
    unsigned long long lab;
    uint64_t adj;
    uint32_t idx;
};

// ---- graph preparation
cudaError_t launch_validate(const DevGraph &g, int32_t num_labels, int *err, cudaStream_t st);
cudaError_t launch_prepare(const DevGraph &g, int64_t *piece_cnt, int32_t *end_off, int32_t *rank,
                           int32_t *cls_size, cudaStream_t st);

// ---- neighbour-adjacency matrices of vertices of degree >= dmin (DevGraph::tri_off):
//      words[v] = d * ceil(d / 32) or 0; then, with off = exclusive prefix of words, the bits
//      and tri_off (-1 for vertices without a matrix); bits must be zeroed first
#define FSM_TRI_DMIN 32
#define FSM_TRI_BUDGET ((int64_t)512 << 20)   // bytes
cudaError_t launch_tri_words(const DevGraph &g, int32_t dmin, int64_t *words, cudaStream_t st);
cudaError_t launch_tri_bits(const DevGraph &g, int32_t dmin, const int64_t *off, int64_t *tri_off, uint32_t *bits,
                            cudaStream_t st);

// ---- scans (exclusive, out has n+1 entries, out[n] = total)
size_t scan_temp_bytes(int64_t n);
cudaError_t launch_scan_i64(const int64_t *in, int64_t *out, int64_t n, void *temp, cudaStream_t st);

// ---- per-batch unit piece counts: cnt[u] = g.ppc[v] for the key vertex v = fv[(u % L) * fN + e0 + u / L],
//      with the centre pairs cut to centre_pairs(d, c) when L == 2 (see fsm_device.cuh); with
//      V = FSM_EXPLORE_SV (single-vertex exploration) cnt[u] = d(v); with V = FSM_EXPLORE_TV_QUOTA
//      the count is cut to min(c, quota), and at L == 2 to 0 for edges outside their key vertex's
//      edge quota (see fsm_device.cuh)
cudaError_t launch_unit_counts(const DevGraph &g, const int32_t *fv, int64_t fN, int64_t e0, int64_t ne, int L, int V,
                               int64_t quota, int64_t edge_quota, uint64_t qseed, int64_t *cnt, cudaStream_t st);

// algorithmic bytes of one batch of units, added to *sum: per unit 4 * (d(v) + end pieces of v)
// (the key list and every end list read once; single-vertex exploration: 4 * d(v)) plus
// 4 * (L + 1) per embedding (vertices + id)
cudaError_t launch_unit_bytes(const int32_t *row_ptr, const int64_t *piece_cnt, const int32_t *fv, int64_t fN,
                              int64_t e0, int64_t ne, int L, int V, unsigned long long *sum, cudaStream_t st);

// Group a stored frontier by pattern id: offsets = exclusive prefix of counts[P] (P+1 entries),
// then every embedding is copied to off[pid] + (arrival order within its pattern).
cudaError_t launch_group_by_pattern(const int32_t *fv, const int32_t *fpid, int64_t N, int L, const int64_t *off,
                                    unsigned long long *cursor, int32_t *out_v, int32_t *out_pid, cudaStream_t st);
cudaError_t launch_u64_to_i64(const unsigned long long *in, int64_t *out, int64_t n, cudaStream_t st);

// ---- quick-pattern table
cudaError_t launch_fill_u64(unsigned long long *p, unsigned long long v, int64_t n, cudaStream_t st);
cudaError_t launch_qp_compact(const unsigned long long *keys, int64_t cap, int64_t *slots,
                              unsigned long long *n_out, cudaStream_t st);
// canonical code of each distinct key; writes recs[q] (idx = q) and perm[slot]
cudaError_t launch_qp_canon(int L, int V, const unsigned long long *keys, const int64_t *slots, int64_t nq,
                            const uint64_t *pat_lab8, const uint64_t *pat_adj8, CodeRec *recs,
                            uint64_t *perm, cudaStream_t st);
// sort recs[0..n) ascending by (lab, adj, idx); recs must have room for next_pow2(n) entries
cudaError_t launch_sort_codes(CodeRec *recs, int64_t n, cudaStream_t st);
// after sorting: pattern ids.  flags/ids scratch of n+1 entries.  Writes qp_pattern[slot],
// pattern codes pat_lab/pat_adj, and *n_pat.
cudaError_t launch_assign_patterns(const CodeRec *recs, int64_t n, const int64_t *slots, int64_t *flag,
                                   int64_t *ids, void *scan_tmp, int32_t *qp_pattern,
                                   unsigned long long *pat_lab, uint64_t *pat_adj, cudaStream_t st);
// per pattern: orbit word (representative per canonical position), smallest orbit size
cudaError_t launch_orbits(int K, const unsigned long long *pat_lab, const uint64_t *pat_adj, int64_t np,
                          uint64_t *orbit, int32_t *min_orbit, cudaStream_t st);
// pattern embedding counts: pat_count[pattern[slot]] += count[slot]
cudaError_t launch_pattern_counts(const int64_t *slots, int64_t nq, const int32_t *qp_pattern,
                                  const unsigned long long *qp_count, unsigned long long *pat_count,
                                  cudaStream_t st);
// live patterns (count * smallest orbit >= t) and the words of each orbit bitmap
cudaError_t launch_domain_sizes(int K, const unsigned long long *pat_lab, const uint64_t *orbit,
                                const int32_t *min_orbit, const unsigned long long *pat_count,
                                int64_t np, int64_t t, const int32_t *cls_size, uint8_t *live,
                                int64_t *words, cudaStream_t st);
// offsets from the scanned sizes (-1 where no bitmap)
cudaError_t launch_domain_offsets(const int64_t *words, const int64_t *scanned, int64_t n8, int64_t *off,
                                  cudaStream_t st);
// MNI support: sigma[P] = min over orbit bitmaps of popcount (0 for non-live patterns)
cudaError_t launch_support(int K, const uint64_t *orbit, const uint8_t *live, const int64_t *dom_off,
                           const int64_t *words, const uint32_t *dom, int64_t np,
                           unsigned long long *sigma, cudaStream_t st);
// frequent flags (sigma >= t) as int64 0/1 for scanning, and the new ids afterwards
cudaError_t launch_freq_flags(const unsigned long long *sigma, int64_t np, int64_t t, int64_t *flag,
                              cudaStream_t st);
cudaError_t launch_new_ids(const int64_t *flag, const int64_t *scanned, int64_t np, int32_t *newid,
                           cudaStream_t st);
// gather frequent patterns: codes, sigma, counts -> compact arrays; also level tables (lab8/adj8)
cudaError_t launch_gather_frequent(int K, const int32_t *newid, int64_t np, const unsigned long long *pat_lab,
                                   const uint64_t *pat_adj, const unsigned long long *sigma,
                                   const unsigned long long *pat_count, unsigned long long *o_lab,
                                   uint64_t *o_adj, unsigned long long *o_sigma, unsigned long long *o_count,
                                   uint64_t *o_lab8, uint64_t *o_adj8, cudaStream_t st);
// sum of counts of frequent patterns (the next frontier's size)
cudaError_t launch_sum_frequent(const int32_t *newid, const unsigned long long *pat_count, int64_t np,
                                unsigned long long *sum, cudaStream_t st);

// ---- base levels
// level 1: frequent labels (cls_size >= t): flag per label
// level 1 frontier: vertices whose label is frequent (deterministic compaction)
cudaError_t launch_level1_frontier(const DevGraph &g, const int32_t *label_newid, int64_t *flag,
                                   int64_t *scanned, void *scan_tmp, int32_t *fv, int32_t *fpid,
                                   cudaStream_t st);
// level 2: edge patterns over label pairs (lo <= hi) indexed lo*NL + hi
cudaError_t launch_level2_domains(const DevGraph &g, int32_t NL, const int64_t *pair_off,
                                  uint32_t *dom, unsigned long long *pair_count, cudaStream_t st);
cudaError_t launch_level2_offsets(int32_t NL, const int32_t *cls_size, int64_t *pair_off,
                                  int64_t *total_words, cudaStream_t st);
cudaError_t launch_level2_support(int32_t NL, const int32_t *cls_size, const int64_t *pair_off,
                                  const uint32_t *dom, unsigned long long *sigma, cudaStream_t st);
// level 2 frontier: every edge of a frequent pair in canonical order
cudaError_t launch_level2_frontier(const DevGraph &g, int32_t NL, const int32_t *pair_newid,
                                   int64_t *flag, int64_t *scanned, void *scan_tmp, int32_t *fv,
                                   int64_t fN, int32_t *fpid, cudaStream_t st);

// size-1 and size-2 pattern tables (single-block kernels over the <= 64 labels / label pairs):
// frequent ids in code order, level tables, codes, supports, counts; *n_freq = frequent count
cudaError_t launch_level1_tables(int32_t NL, const int32_t *cls_size, int64_t t, int32_t *label_newid,
                                 uint64_t *lab8, uint64_t *adj8, unsigned long long *clab, uint64_t *cadj,
                                 unsigned long long *sigma, unsigned long long *count,
                                 unsigned long long *n_freq, cudaStream_t st);
cudaError_t launch_level2_tables(int32_t NL, const unsigned long long *pair_sigma,
                                 const unsigned long long *pair_count, int64_t t, int32_t *pair_newid,
                                 uint64_t *lab8, uint64_t *adj8, unsigned long long *clab, uint64_t *cadj,
                                 unsigned long long *sigma, unsigned long long *count,
                                 unsigned long long *n_freq, cudaStream_t st);

// number of kernels launched by this process so far
int64_t launches_so_far();
void note_launches(int64_t n);

// ---- sampled final level
// Lists of the kept directed edges (v -> a kept iff keep_edge(seed, thr, v, a)): counts, then
// (after an exclusive scan into prow64) the lists, the end-piece prefixes and piece counts.
cudaError_t launch_sample_count(const DevGraph &g, uint64_t seed, uint64_t thr, int64_t *cnt, cudaStream_t st);
cudaError_t launch_sample_lists(const DevGraph &g, uint64_t seed, uint64_t thr, const int64_t *prow64, int32_t *prow,
                                int32_t *pcol, int32_t *pend, int64_t *ppc, cudaStream_t st);
// by_rank[cls_off[l] + rank[v]] = v for every vertex v of label l (cls_off: exclusive prefix of
// class sizes, computed by the kernel itself)
cudaError_t launch_by_rank(const DevGraph &g, int32_t NL, const int32_t *cls_size, int64_t *cls_off,
                           int32_t *by_rank, cudaStream_t st);
// The 32 features of every candidate pattern of a sampled level (layout in fsm_api.cu):
//   [0..8)   log1p of the sampled domain popcount of each orbit, ascending, zero-padded
//   [8..16)  log(|V_l| / n) of the label of each canonical position, zero-padded
//   [16..24) mean log1p(degree) over the sampled domain of each canonical position's orbit
//   [24..32) k, edges, log p, log1p(sampled embeddings), log(t / n), log |Aut|,
//            log((smallest popcount + 1) / p), log n
cudaError_t launch_features(int K, const unsigned long long *pat_lab, const uint64_t *pat_adj, const uint64_t *orbit,
                            const int64_t *dom_off, const int64_t *words, const uint32_t *dom,
                            const unsigned long long *pat_count, const int32_t *cls_size, const int64_t *cls_off,
                            const int32_t *by_rank, const int32_t *row_ptr, int32_t n, double p, int64_t t,
                            int64_t np, const int64_t *aut, float *feat, cudaStream_t st);
// Automorphism group size of each pattern (the orbits kernel enumerates the same orders)
cudaError_t launch_aut_size(int K, const unsigned long long *pat_lab, const uint64_t *pat_adj, int64_t np,
                            int64_t *aut, cudaStream_t st);

// Exact recount of sampled mining: for every pattern with uncertain[P], every dissection of
// its canonical graph into a connected 3-vertex part and a connected (K-2)-vertex part sharing
// one vertex: mark the part's size-(K-2) pattern (its id found by binary search among the
// sorted codes s_lab/s_adj of the stored level) in need_s and the piece in need_piece.
cudaError_t launch_needed_parts(int K, const unsigned long long *lab, const uint64_t *adj, const uint8_t *uncertain,
                                int64_t np, const unsigned long long *s_lab, const uint64_t *s_adj, int64_t s_np,
                                uint8_t *need_s, uint8_t *need_piece, cudaStream_t st);
// keep the stored embeddings whose pattern is flagged: out has room for N rows
cudaError_t launch_compact_frontier(const int32_t *fv, const int32_t *fpid, int64_t N, int L, const uint8_t *keep,
                                    int64_t *flag, int64_t *scanned, void *scan_tmp, int32_t *out_v, int64_t outN,
                                    int32_t *out_pid, cudaStream_t st);
cudaError_t launch_flag_count(const int32_t *fpid, int64_t N, const uint8_t *keep, int64_t *flag, cudaStream_t st);
cudaError_t launch_and_u8(uint8_t *a, const uint8_t *b, int64_t n, cudaStream_t st);
// out[P] = keep[P] ? count[P] : 0
cudaError_t launch_keep_counts(const unsigned long long *count, const uint8_t *keep, int64_t np, unsigned long long *out,
                               cudaStream_t st);

// decision of sampled mining with a model: pred = predicted log support; keep[P] = 1 when
// pred >= logt + delta, uncertain[P] = 1 when |pred - logt| <= delta (strictly inside: below
// logt + delta)
cudaError_t launch_decide(const float *pred, int64_t np, float logt, float delta, uint8_t *keep, uint8_t *uncertain,
                          cudaStream_t st);

// *out = the device's global timer (ns), in stream order: the start of a call's time limit
cudaError_t launch_stamp_time(unsigned long long *out, cudaStream_t st);

// MNI supports from the one-pass last level: sigma[P] = the smallest orbit popcount of pattern
// P's bitmap block, found through its entry in the code table (ckeys / coff, cmask + 1 slots)
cudaError_t launch_fused_support(int K, const unsigned long long *plab, const uint64_t *padj, const uint64_t *orbit,
                                 int64_t np, const unsigned long long *ckeys, const unsigned long long *coff,
                                 uint64_t cmask, const int32_t *cls_size, const uint32_t *pool, unsigned long long *sigma,
                                 cudaStream_t st);

// Domain pass helper: for every distinct key (slot) and local position h, the word offset of
// the bitmap its vertex goes to (the orbit of canonical position perm[h] of its pattern), or -1
// when the pattern has no domains.
cudaError_t launch_slot_bases(int K, const int64_t *slots, int64_t nq, const int32_t *qp_pattern,
                              const uint64_t *qp_perm, const uint8_t *live, const uint64_t *orbit,
                              const int64_t *dom_off, int64_t *slot_base, cudaStream_t st);

// ---- pieces: mark the frequent size-3 patterns by piece index
cudaError_t launch_piece_table(const unsigned long long *lab, const uint64_t *adj, int64_t n,
                               uint8_t *piece_freq, cudaStream_t st);

} // namespace fsm
