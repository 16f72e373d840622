/*
 * fsm.h -- C ABI of the GB300 frequent-subgraph-mining library (two-vertex exploration).
 *
 * The library finds every size-k pattern of one labeled, undirected input graph whose MNI
 * support is at least t (the FSM problem of Section 2.2).  Mining runs level by level
 * (sizes 1 -> 3 -> 5 -> 7 -> 9 for odd k, 2 -> 4 -> 6 -> 8 for even k): every embedding of every
 * frequent size-l pattern is joined with every frequent size-3 subgraph (wedge or triangle)
 * that shares exactly one vertex with it (two-vertex exploration, Section 4.1, Theorem 1),
 * duplicates are removed by smallest-vertex-first dissection (Section 4.3, Algorithm 1),
 * joins whose joining-point triples form an infrequent size-3 pattern are pruned
 * (Section 4.5), results are grouped by index-based quick pattern (Section 4.4) and each
 * distinct quick pattern is canonicalised once; MNI support (Definition 2) is aggregated in
 * per-pattern, per-orbit domain bitmaps.  Every step runs in this library's CUDA kernels on
 * one GPU; nothing here falls back to the CPU.
 *
 * Conventions shared by every entry point:
 *   - Return value: FSM_OK (0) or a negative FSM_E* code; fsm_last_error() then holds a
 *     thread-local message.  On error, every out-pointer is left NULL / untouched.
 *   - Pointers passed in are HOST pointers unless the name says otherwise; the library
 *     copies what it needs and never keeps or frees caller memory.
 *   - A graph handle owns device memory until fsm_free_graph(); a result handle owns host
 *     memory until fsm_free_result().  Handles are not thread-safe: one thread per handle.
 *   - Vertex ids are int32 in [0, n); labels are int32 in [0, num_labels), num_labels <= 64.
 *   - Pattern encoding (output): labels[k] in canonical order, and the canonical edges as
 *     adj_bits (k <= 8) with bit (i*k + j), LSB = bit 0, set for every canonical edge i < j, or
 *     as pair bits (any k <= 9; fsm_result_pairs) with bit q set when the q-th pair of
 *     (0,1), (0,2), ..., (k-2,k-1) is an edge.  The canonical form of a labeled graph is the
 *     lexicographically smallest (label sequence, adjacency sequence A(0,1), A(0,2), ...,
 *     A(k-2,k-1)) over all vertex orders; results are sorted ascending by that same (label
 *     sequence, adjacency sequence) key.
 */
#ifndef FSM_H
#define FSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    FSM_OK = 0,
    FSM_EINVAL = -1,        /* bad argument or malformed CSR */
    FSM_ENOMEM = -2,        /* a device or host allocation failed */
    FSM_ECUDA = -3,         /* a CUDA runtime call or kernel failed */
    FSM_ETIMEOUT = -4,      /* a bounded device loop gave up (see fsm_last_error) */
    FSM_EUNSUPPORTED = -5   /* input or request outside the supported range */
};

typedef struct fsm_graph fsm_graph;
typedef struct fsm_result fsm_result;
typedef struct fsm_mlp fsm_mlp;

/*
 * fsm_load_graph -- copy one labeled graph G = (V, E, L) (Section 2.1) to the current CUDA
 * device and prepare it for mining.
 *   row_ptr  int32[n+1], row_ptr[0] = 0, nondecreasing; row_ptr[n] = 2|E| = nnz.
 *   col      int32[nnz]: the neighbours of v are col[row_ptr[v] .. row_ptr[v+1]), sorted
 *            strictly ascending; every undirected edge appears in both directions; no
 *            self-loops, no duplicates.
 *   labels   int32[n]: vertex labels in [0, num_labels).
 *   n >= 1, 1 <= num_labels <= 64.
 * The CSR is validated on the device (sortedness, symmetry, self-loops, duplicates, label
 * range): a malformed graph gives FSM_EINVAL.  nnz >= 2^31 gives FSM_EUNSUPPORTED.
 * Ownership: the arrays are copied; *out owns device memory until fsm_free_graph().
 */
int fsm_load_graph(const int32_t *row_ptr, const int32_t *col, const int32_t *labels,
                   int32_t n, int32_t num_labels, fsm_graph **out);

/*
 * fsm_set_option -- set a per-graph option (takes effect on the next fsm_mine call).
 *   "mode"       0 = edge-induced embeddings (default; the experiments' setting, Section 6.1),
 *                1 = vertex-induced embeddings (Section 2.1).
 *   "stream"     a cudaStream_t (cast to int64) that all later work of this graph is issued on;
 *                0 restores the library's own stream.  The caller keeps ownership.
 *   "launch"     0 = one launch per frontier batch of at most "batch" embeddings, sized on
 *                the host (default); 1 = one persistent work-stealing launch per pass over the
 *                whole frontier, all sizes kept on the device, captured with its prefix kernels
 *                in a CUDA graph (its per-unit piece prefix takes 8 bytes per embedding and key
 *                position; a frontier whose prefix would exceed a quarter of the free device
 *                memory is split into the fewest equal ranges that fit, one launch each, in the
 *                same graph); 2 = one launch per frontier
 *                pattern (the frontier grouped by pattern id), captured in one CUDA graph.  All
 *                modes give identical results.
 *   "group"      with launch 1: 1 = group the frontier by pattern id before each level (as
 *                launch 2 does), 0 = keep emission order, 2 = group frontiers of size >= 3 and
 *                keep the order of edges (default).  Results are identical.
 *   "autotune"   1 = on the first call per level, time the domain pass on 1/32 of the
 *                frontier for chunk sizes 256, 1024, 4096, 16384 and keep the fastest for later
 *                passes and calls (reported as stat "chunk_l<l>"); 0 = forget tuned values.
 *   "chunk"      pieces per work-stealing chunk (power of two, 32..65536; 0 = default: the largest
 *                power of two from 256 to 16384 that leaves at least 64 chunks per warp and spans
 *                at most about 16 units' pieces).
 *   "batch"      frontier embeddings per batch (>= 1024; 0 = default).
 *   "explore"    0 = two-vertex exploration (default, Section 4.1); 1 = single-vertex
 *                exploration, l -> l+1 (the ablation Section 6 compares against): every level
 *                joins each stored embedding with one neighbour of a key vertex, a new embedding
 *                is kept when its new vertex is the largest-id vertex whose removal leaves it
 *                connected and its key vertex is that vertex's smallest-id neighbour in the
 *                embedding; no size-3 pruning table.  Exact results, identical to 0; k <= 7.
 *   "quick_pattern" 0 = index-based quick patterns (default, Section 4.4); 1 = edge-list quick
 *                patterns (the baseline Section 6 compares against): each accepted join is keyed
 *                by its labels and edges listed over its vertices in ascending id order, so more
 *                distinct keys are canonicalised (stat "quick_patterns").  Identical results;
 *                k <= 7.
 *   "join_quota" ST x of Section 5 (0 = off, default): every join l -> l+2 runs at most x^2
 *                candidate pieces per key group (stored embedding s, key vertex v) and, when
 *                edges are joined (l = 2), at most x edges per key vertex; candidates are drawn
 *                by an affine progression seeded from option "seed" and the ids of s and v (see
 *                the quota notes in the library's device header).  Supports and counts are those
 *                of the drawn embeddings, lower bounds of the exact ones (fsm_result_exact = 0),
 *                and every level keeps the patterns whose drawn support reaches t.
 *   "match_quota" M.ST of Section 5 (0 = off, default): the size-3 level runs at most this many
 *                candidate pieces per vertex (candidates whose smallest vertex is not that
 *                vertex are dropped after the draw).  Quotas exclude "explore" = 1,
 *                "quick_pattern" = 1 and sample_rate < 1.
 *   "qp_capacity" slots of the first quick-pattern hash table of every level (power of two,
 *                64..2^30; 0 = at least 2^20, sized from the previous call).  A table that fills
 *                past half is grown x4 and its pass repeated (stat "qp_grows"); results are
 *                identical.
 *   "fused"      1 = the last level of exact mining (k <= 7) is enumerated once: each accepted
 *                join is counted under its quick pattern and sets its MNI domain bits at once;
 *                the first lane to meet a quick pattern canonicalises it and claims its
 *                pattern's orbit bitmaps (every pattern gets bitmaps, frequent or not); 0 = a
 *                count pass, canonicalisation, then a domain pass for the patterns that can
 *                still reach t (default).  Identical results; when the bitmap pool or the pattern
 *                table runs out, the level is counted again and finished in two passes (stat
 *                "fused_fallbacks").
 *   "fused_pool" size in 32-bit words of the one-pass level's bitmap pool (0 = twice what the
 *                previous call used, else 40% of the free device memory).
 *   "seed"       64-bit seed of the piece sampling of fsm_mine with sample_rate < 1 (default 0).
 *   "candidates" 1 = sampled mining returns every candidate pattern of the sampled level with
 *                its estimated support (smallest orbit popcount / p) and its 32 features
 *                (fsm_result_features), deciding nothing; 0 = decide (default).
 *   "model"      an fsm_mlp* (cast to int64) that sampled mining uses to predict supports; 0 =
 *                none (sampled mining then keeps patterns whose estimate reaches t).  The graph
 *                borrows the network; keep it alive while the graph uses it.
 *   "delta_milli" recount band of sampled mining with a model, in thousandths of a natural log
 *                unit (default 500): patterns with |log prediction - log t| <= delta are
 *                recounted exactly.
 *   "debug"      1 = the extension kernels check every decoded list index against its list
 *                before reading; a failed check sets the call's error word and skips the read (no
 *                trap), and the call returns FSM_ECUDA; 0 = off (default).
 *   "time_limit_ms" > 0: the extension kernels stop taking work once this much device time has
 *                passed since the call started (checked at every work chunk) and the call returns
 *                FSM_ETIMEOUT with no result; the handle stays usable; 0 = no limit (default).
 *   "fail_alloc_after" test hook: > 0 makes the call's n-th device allocation report failure, so
 *                the call returns FSM_ENOMEM (everything it allocated is released); 0 = off.
 *   "profile"    1 = time every extension-kernel launch with CUDA events and sum its algorithmic
 *                bytes (reported by fsm_result_stat); adds one synchronisation per launch.
 * Unknown keys or out-of-range values give FSM_EINVAL.
 */
int fsm_set_option(fsm_graph *g, const char *key, int64_t value);

/*
 * fsm_mine -- every pattern with exactly k vertices and MNI support >= min_support
 * (Section 2.2 problem statement; Definition 2).
 *   1 <= k <= 9, min_support >= 1, sample_rate in (0, 1]; 1.0 means exact mining.  k = 9
 *   (Section 6 mines 9-vertex patterns) runs with two-vertex exploration and index-based quick
 *   patterns, exactly or with sampling quotas; the single-vertex and edge-list ablations stop
 *   at k = 7 and rate-sampled mining at k = 8 (FSM_EUNSUPPORTED above).
 * Exact mining (sample_rate = 1) returns exact MNI supports and embedding counts.
 * Sampled mining (sample_rate = p < 1, k >= 3; Section 5's subgraph sampling, here at a rate
 * instead of a per-key quota): every level but the last is mined exactly; in the last level a
 * directed edge x -> y is kept iff splitmix64(splitmix64(splitmix64(seed) ^ x) ^ y) <
 * floor(sqrt(p) * 2^64) (seed from option "seed"), and only pieces made of kept edges seen
 * from the joining vertex v are enumerated: {v; a, b} with v -> a and v -> b kept, v - a - b
 * with v -> a and a -> b kept, about p of all pieces.  Each candidate pattern's
 * support is then decided by the model (option "model"): predictions above t * e^delta are
 * kept with the predicted support (clamped between the sampled support, a lower bound, and the
 * smallest label class of the pattern, an upper bound), predictions within the band are recounted exactly by an
 * exact last level restricted to the parts those patterns can be dissected into, the rest are
 * dropped.  Without a model the estimate (smallest sampled orbit popcount) / p decides.
 * fsm_result_exact tells which supports were counted exactly.
 * Ownership: *out is a host-side result owned by the caller until fsm_free_result().
 */
int fsm_mine(fsm_graph *g, int32_t k, int64_t min_support, double sample_rate,
             fsm_result **out);

/* Number of patterns in a result (>= 0), or FSM_EINVAL for a NULL result. */
int64_t fsm_result_count(const fsm_result *r);

/*
 * fsm_result_get -- pattern i (0 <= i < count) of a result.
 *   labels_k  int32[k] written with the canonical labels (may be NULL).
 *   adj_bits  bit (i*k + j) set per canonical edge i < j (may be NULL); k <= 8 only: a k = 9
 *             result gives FSM_EUNSUPPORTED for a non-NULL adj_bits (use fsm_result_pairs).
 *   support   MNI support (may be NULL).
 */
int fsm_result_get(const fsm_result *r, int64_t i, int32_t *labels_k, uint64_t *adj_bits,
                   int64_t *support);

/* Number of embeddings (subgraphs, not maps) of pattern i, counted during mining. */
int fsm_result_embeddings(const fsm_result *r, int64_t i, int64_t *count);

/*
 * fsm_result_copy -- all patterns at once: labels int32[count*k] (row-major), adj_bits
 * uint64[count] (k <= 8 only, as in fsm_result_get), support int64[count], embeddings
 * int64[count]; any pointer may be NULL.
 */
int fsm_result_copy(const fsm_result *r, int32_t *labels, uint64_t *adj_bits, int64_t *support,
                    int64_t *embeddings);

/*
 * fsm_result_pairs -- the canonical edges of every pattern as pair bits, for any k <= 9:
 * pairs[i] (uint64[count]) has bit q set when the q-th pair of (0,1), (0,2), ..., (k-2,k-1)
 * (row-major, q from 0) is an edge of pattern i.  FSM_EINVAL for NULL arguments.
 */
int fsm_result_pairs(const fsm_result *r, uint64_t *pairs);

/*
 * fsm_result_exact -- exact[i] = 1 when pattern i's support and count were counted exactly, 0
 * when they are estimates of sampled mining (int32[count]).
 */
int fsm_result_exact(const fsm_result *r, int32_t *exact);

/*
 * fsm_result_features -- the 32 features of every pattern (float[count * 32], row-major) of a
 * sampled mining call made with option "candidates" = 1; FSM_EINVAL otherwise.  Features:
 * [0..8) log1p of each orbit's sampled domain popcount, ascending, zero-padded; [8..16)
 * log(|V_l| / n) for each canonical position's label; [16..24) mean log1p(degree) over the
 * sampled domain of each position's orbit; [24..32) k, number of edges, log p,
 * log1p(sampled embeddings), log(t / n), log |Aut|, log((smallest popcount + 1) / p), log n.
 */
int fsm_result_features(const fsm_result *r, float *features);

/*
 * fsm_result_stat -- a run counter of the mining call that made r:
 *   "k", "levels", "pieces" (size-3 pieces enumerated by the count passes; "pieces_l<l>" per
 *   extended level size l = 1..7), "candidates" (joins
 *   tested), "embeddings" (accepted joins, all levels),
 *   "final_embeddings" (accepted joins of the last level), "qp_grows" (quick-pattern table
 *   overflows, each a grown table and a repeated pass), "fused_fallbacks" (one-pass last levels
 *   redone in two passes), "fused_pool_words" (bitmap pool words the one-pass level used),
 *   "quick_patterns" (distinct index
 *   based quick patterns, i.e. canonicalisations, all levels), "patterns" (distinct patterns
 *   of the last level), "live_patterns" (last-level patterns given a domain),
 *   "frontier_max" (largest stored level), "kernel_launches", "time_ns" (device time of the
 *   whole call, CUDA events), "final_level_ns" (device time of the last level); with the
 *   "profile" option also, per extension pass P in {count, domain, emit}: "P_ns" (summed
 *   launch durations), "P_launches", "P_bytes" (algorithmic bytes: 4 * (d(v) + end pieces of v)
 *   per (embedding, key position) unit, 4 * (l + 1) per embedding read, for domain also
 *   4 * (l + 2) per accepted join of a pattern given a domain (one bitmap word per position),
 *   and for emit 4 * (l + 3) per embedding written), and the same per extended level size l as
 *   "P_ns_l<l>", "P_launches_l<l>", "P_bytes_l<l>" (l = 1..7); "chunk_l<l>" (autotuned chunk
 *   size of level l, 0 if none).  In launch modes 1 and 2 a pass's time covers its CUDA graph
 *   (the prefix-sum kernels included).
 */
int fsm_result_stat(const fsm_result *r, const char *key, int64_t *value);

void fsm_free_result(fsm_result *r);
void fsm_free_graph(fsm_graph *g);

/* Message of the last failing call on this thread ("" if none). */
const char *fsm_last_error(void);

/*
 * Support-prediction network of sampled mining (no counterpart in the paper): a 32 -> 64 ->
 * 64 -> 1 multilayer perceptron with ReLU, inputs standardised by stored means and deviations,
 * BF16 weights in every product with FP32 accumulation, FP32 master weights trained by Adam
 * on the mean squared error of log(MNI support).  Parameters (6337 floats, FP32): W1[32][64]
 * (input, unit), b1[64], W2[64][64], b2[64], w3[64], b3.  Host pointers unless named d_*.
 *   fsm_mlp_create       He-uniform weights from a splitmix64 stream of seed; zero biases.
 *   fsm_mlp_set_params / fsm_mlp_get_params   copy the 6337 master weights in / out (set also
 *                        resets Adam's moments).
 *   fsm_mlp_set_norm     input means and standard deviations (32 each, deviations > 0).
 *   fsm_mlp_fit_norm     the same, computed on the device from X[n][32]: column means and
 *                        population standard deviations (accumulated in double), deviations
 *                        floored at 1e-3.
 *   fsm_mlp_gradients    mean squared error over X[n][32], Y[n] and its gradient (6337 floats).
 *   fsm_mlp_train        epochs of shuffled minibatches (order from a splitmix64 stream of seed),
 *                        Adam (beta 0.9, 0.999, eps 1e-8) at rate lr; final_loss = last epoch's
 *                        mean squared error.
 *   fsm_mlp_predict      outputs (predicted log support) for X[n][32].
 *   fsm_mlp_predict_device the same on device arrays, on stream.
 */
int fsm_mlp_create(uint64_t seed, fsm_mlp **out);
int fsm_mlp_set_params(fsm_mlp *m, const float *params);
int fsm_mlp_get_params(const fsm_mlp *m, float *params);
int fsm_mlp_set_norm(fsm_mlp *m, const float *mean, const float *stdev);
int fsm_mlp_fit_norm(fsm_mlp *m, const float *X, int64_t n);
int fsm_mlp_gradients(fsm_mlp *m, const float *X, const float *Y, int64_t n, float *grads, float *loss);
int fsm_mlp_train(fsm_mlp *m, const float *X, const float *Y, int64_t n, int32_t epochs, int32_t batch,
                  float lr, uint64_t seed, float *final_loss);
int fsm_mlp_predict(const fsm_mlp *m, const float *X, int64_t n, float *out);
int fsm_mlp_predict_device(const fsm_mlp *m, const float *d_X, int64_t n, float *d_out, void *stream);
void fsm_mlp_free(fsm_mlp *m);

/*
 * fsm_debug_dissect -- host build of the library's smallest-vertex-first dissection
 * (Section 4.3, Algorithm 1, function dissect with n = 3) on one connected subgraph:
 *   k (4..8) vertices with global ids ids[k] (distinct), adjacency rows adj[k] (bit j of
 *   adj[i] set when i ~ j).  Writes the 3-vertex part as a bit mask over the k local indices
 *   (*l_mask) and the shared vertex's local index (*join).  Returns FSM_OK, or
 *   FSM_EINVAL if the input is not a connected simple graph.  *used_fallback is 1 when the
 *   greedy rule found no dissection and the exhaustive rule answered instead.  Test hook only.
 */
int fsm_debug_dissect(int32_t k, const int32_t *ids, const uint32_t *adj, uint32_t *l_mask,
                      int32_t *join, int32_t *used_fallback);

/*
 * fsm_edge_supports_noalloc -- MNI support and embedding count of every labeled edge pattern
 * (the size-2 level), computed without allocating any device memory.  The paper has no
 * counterpart; this entry point exists for callers that cannot call cudaMalloc, such as code
 * that runs inside an allocator's own callback, or a process whose device memory is fully
 * reserved by another framework's pool.
 *   d_row_ptr, d_col, d_labels  DEVICE pointers to a CSR in the layout of fsm_load_graph
 *                              (validated on the device before any other read: row_ptr[0]
 *                              = 0, every row range inside [0, row_ptr[n]] and nondecreasing,
 *                              rows sorted and symmetric, labels in range; malformed input
 *                              gives FSM_EINVAL).  d_col must hold row_ptr[n] entries.
 *   n >= 1, 1 <= num_labels <= 64.
 *   d_support, d_count          DEVICE uint64[num_labels * num_labels] written by the call:
 *                              entry lo * num_labels + hi (lo <= hi) holds the MNI support and
 *                              the edge count of the pattern with labels (lo, hi); entries with
 *                              hi < lo are 0.  fsm_mine(k = 2) returns the same supports and
 *                              counts for the pairs whose support reaches its threshold.
 *   stream                      cudaStream_t to run on (NULL = the default stream).  Every
 *                              call copies row_ptr[n] and the validation flag back to the host
 *                              and synchronises this stream, twice, before it returns.
 * Scratch: one static device array of 64 MiB, reserved when the library's device code is
 * loaded on a GPU and kept until the process exits; no cudaMalloc, cudaFree or allocating
 * library routine is called.  A graph whose scratch need, about 4 * (n + num_labels *
 * (n / 32 + num_labels) + 6 * num_labels^2) bytes, exceeds the array is rejected with
 * FSM_EUNSUPPORTED (and a message giving both sizes) before any device work.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  Every call reuses the same array and clears the part it
 * needs: calls that overlap on the GPU (other threads, other streams) race and must not be
 * issued.
 */
int fsm_edge_supports_noalloc(const int32_t *d_row_ptr, const int32_t *d_col, const int32_t *d_labels,
                              int32_t n, int32_t num_labels, uint64_t *d_support, uint64_t *d_count,
                              void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FSM_H */
