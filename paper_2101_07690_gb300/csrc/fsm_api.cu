// fsm_api.cu -- the C ABI (include/fsm.h) and the host-side level loop.
//
// Level loop (Section 3 workflow, generalised level by level):
//   size 1   label classes; MNI of a one-vertex pattern is its class size;
//   size 2   labeled edge patterns with per-orbit domain bitmaps;
//   size 3   two-vertex extension of every size-1 embedding (each connected size-3 subgraph is
//            produced once, keyed at its smallest vertex); its frequent patterns are the pieces
//            of every later join and the table of the joining-point pruning (Section 4.5);
//   l -> l+2 two-vertex extension of the stored frequent size-l embeddings (odd k from size 3,
//            even k from size 2), three passes over the same enumeration: count quick patterns,
//            fill MNI domains of patterns that can still reach the threshold, and (non-final
//            levels) emit the embeddings of frequent patterns in canonical order.
// Between passes, each distinct quick pattern is canonicalised once (Section 4.4) and the
// canonical codes are sorted so pattern ids are deterministic.
#include "fsm.h"
#include "fsm_extend.cuh"
#include "fsm_kernels.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

using namespace fsm;

namespace {

thread_local std::string g_last_error;

struct FsmError {
    int code;
    std::string msg;
};

[[noreturn]] void fail(int code, const std::string &msg) { throw FsmError{code, msg}; }

void ck(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        fail(FSM_ENOMEM, std::string(what) + ": " + cudaGetErrorString(e));
    }
    fail(FSM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int set_error(const FsmError &e) {
    g_last_error = e.msg;
    return e.code;
}

std::once_flag g_pool_once[64];

void keep_pool(int dev) {
    if (dev < 0 || dev >= 64) return;
    std::call_once(g_pool_once[dev], [dev]() {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    });
}

// Stream-ordered device allocations released together.
struct Arena {
    cudaStream_t st;
    std::vector<void *> ptrs;
    int64_t made = 0, fail_at = 0;   // fail_at > 0: the fail_at-th allocation reports failure (test hook)
    explicit Arena(cudaStream_t s) : st(s) {}
    template <class T>
    T *get(int64_t n) {
        void *p = nullptr;
        size_t bytes = (size_t)std::max<int64_t>(n, 1) * sizeof(T);
        bytes = (bytes + 255) & ~(size_t)255;
        if (fail_at > 0 && ++made == fail_at)
            fail(FSM_ENOMEM, "device allocation: injected failure (option fail_alloc_after)");
        ck(cudaMallocAsync(&p, bytes, st), "device allocation");
        ptrs.push_back(p);
        return (T *)p;
    }
    void release(void *p) {
        auto it = std::find(ptrs.begin(), ptrs.end(), p);
        if (it != ptrs.end()) {
            cudaFreeAsync(p, st);
            ptrs.erase(it);
        }
    }
    ~Arena() {
        for (void *p : ptrs) cudaFreeAsync(p, st);
    }
};

template <class T>
T d2h(const T *dptr, cudaStream_t st) {
    T v{};
    ck(cudaMemcpyAsync(&v, dptr, sizeof(T), cudaMemcpyDeviceToHost, st), "copy to host");
    ck(cudaStreamSynchronize(st), "stream synchronize");
    return v;
}

// A CUDA graph captured from a stream.  If an exception leaves the capture open, the
// destructor ends it (so the stream leaves capture mode and later calls see the original error,
// not capture errors) and destroys whatever was captured or instantiated.
struct CapturedGraph {
    cudaStream_t st;
    bool capturing = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    explicit CapturedGraph(cudaStream_t s) : st(s) {}
    void begin() {
        ck(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
        capturing = true;
    }
    void end() {
        capturing = false;
        ck(cudaStreamEndCapture(st, &graph), "end capture");
        ck(cudaGraphInstantiate(&exec, graph, 0), "graph instantiate");
    }
    ~CapturedGraph() {
        if (capturing) {
            cudaGraph_t partial = nullptr;
            cudaStreamEndCapture(st, &partial);
            if (partial) cudaGraphDestroy(partial);
            cudaGetLastError();
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
};

} // namespace

namespace fsm {
// lets other translation units of the C ABI report a message through fsm_last_error()
void set_last_error_message(const std::string &m) { g_last_error = m; }
} // namespace fsm

struct fsm_graph {
    int device = 0;
    int32_t n = 0, NL = 0;
    int64_t nnz = 0;
    cudaStream_t own_stream = nullptr, stream = nullptr;
    int mode = 0, launch = 0, profile = 0;
    int32_t chunk = 0;
    int64_t batch = 0;
    int sms = 0;
    int64_t qp_hint[FSM_MAXL + 1] = {};   // distinct quick patterns seen at each level last time
    int64_t qp_initial = 0;               // option "qp_capacity": first quick-pattern table size (0 = 2^20)
    int explore = 0;                      // option "explore": 0 two-vertex (the method), 1 single-vertex
    int quick_pattern = 0;                // option "quick_pattern": 0 index-based, 1 edge list
    int debug = 0;                        // option "debug": device bounds checks on decoded indices
    int64_t time_limit_ms = 0;            // option "time_limit_ms": FSM_ETIMEOUT past it (0 = none)
    int64_t fail_alloc_after = 0;         // option "fail_alloc_after": injected allocation failure
    int64_t join_quota = 0;               // option "join_quota": ST x of Section 5 (0 = off)
    int64_t match_quota = 0;              // option "match_quota": M.ST of Section 5 (0 = off)
    int autotune = 0;
    int group = 2;   // persistent launch: frontier grouped by pattern id first (1), never (0), from l = 3 (2)
    int fused = 0;
    unsigned long long pool_hint[FSM_MAXL + 1] = {};   // pool words the fused pass used last time
    unsigned long long pool_force = 0;                 // option "fused_pool": fixed pool size
    int32_t tuned_chunk[FSM_MAXL + 1] = {};   // chunk size chosen by the autotuner per level
    // sampled mining
    uint64_t seed = 0;
    int candidates = 0;
    const fsm_mlp *model = nullptr;
    double delta = 0.5;
    int32_t *by_rank = nullptr;
    int64_t *cls_off = nullptr;
    int32_t *row_ptr = nullptr, *col = nullptr, *labels = nullptr, *rank = nullptr, *cls_size = nullptr,
            *end_off = nullptr;
    int64_t *piece_cnt = nullptr;
    int64_t *tri_off = nullptr;   // neighbour-adjacency matrices of high-degree vertices
    uint32_t *tri_bits = nullptr;
    int *err = nullptr;
    unsigned long long *stats = nullptr;   // [0] tested, [1] accepted, [2..] scratch counters
    DevGraph dg() const {
        DevGraph g;
        g.n = n;
        g.nnz = nnz;
        g.row_ptr = row_ptr;
        g.col = col;
        g.labels = labels;
        g.rank = rank;
        g.piece_cnt = piece_cnt;
        g.end_off = end_off;
        g.prow = row_ptr;
        g.pcol = col;
        g.pend = end_off;
        g.ppc = piece_cnt;
        g.tri_off = tri_off;
        g.tri_bits = tri_bits;
        return g;
    }
};

struct fsm_result {
    int k = 0;
    std::vector<int32_t> labels;
    std::vector<uint64_t> adj;           // bit (i*k + j) per canonical edge (k <= 8; 0 for k = 9)
    std::vector<uint64_t> pairs;         // bit q per canonical edge q of (0,1), (0,2), ..., (k-2,k-1)
    std::vector<int64_t> support, count;
    std::vector<int32_t> exact;          // 1: support counted exactly, 0: estimated (sampled mining)
    std::vector<float> features;         // 32 per pattern, sampled mining with "candidates" only
    std::map<std::string, int64_t> stats;
};

namespace {

// Frequent patterns of one level and (optionally) its stored embeddings.
struct LevelSet {
    int L = 0;
    int64_t P = 0;                      // frequent patterns
    uint64_t *lab8 = nullptr, *adj8 = nullptr;
    unsigned long long *clab = nullptr, *sigma = nullptr, *count = nullptr;
    uint64_t *cadj = nullptr;
    int32_t *fv = nullptr, *fpid = nullptr;
    int64_t N = 0;                      // stored embeddings
    float *feat = nullptr;              // sampled level: 32 features per pattern
};

struct RunStats {
    int64_t tested = 0, accepted = 0, pieces = 0, qps = 0, patterns = 0, live = 0, frontier_max = 0, levels = 0,
            final_accepted = 0, launches = 0;
    // profiling (option "profile"): per extension pass, device time, launches, algorithmic bytes
    int64_t recount_patterns = 0, recount_frontier = 0, candidates_sampled = 0, sampled_edges = 0;
    int64_t qp_grows = 0;                  // quick-pattern table overflows (table grown x4, pass repeated)
    int64_t fused_fallbacks = 0;           // one-pass last levels redone as two passes (pool or table full)
    int64_t fused_pool_words = 0;          // bitmap pool words the one-pass last level used
    int64_t pieces_l[FSM_MAXL + 1] = {};   // pieces enumerated by the count pass, per extended level size
    double pass_ns[FSM_MAXL + 1][4] = {};
    int64_t pass_launches[FSM_MAXL + 1][4] = {}, pass_bytes[FSM_MAXL + 1][4] = {};
};

struct Miner {
    fsm_graph *G;
    cudaStream_t st;
    Arena &mem;
    int64_t t;
    RunStats &rs;
    int V = FSM_EXPLORE_TV;   // exploration variant of this call (FSM_EXPLORE_*)

    int grid_for(int L, int pass) {
        int bps = 0;
        cudaError_t e = pass == PASS_COUNT ? occupancy_extend_count(L, V, &bps)
                      : pass == PASS_DOMAIN ? occupancy_extend_domain(L, V, &bps)
                      : pass == PASS_FUSED ? occupancy_extend_fused(L, &bps)
                                            : occupancy_extend_emit(L, V, &bps);
        ck(e, "occupancy query");
        if (bps < 1) bps = 1;
        return G->sms * bps;
    }

    // Profiling records: one event pair per timed region, read after the call's last sync.
    struct ProfEv { cudaEvent_t a, b; int L, pass; };
    std::vector<ProfEv> prof_ev;
    unsigned long long *prof_bytes = nullptr;   // [(FSM_MAXL + 1) * 4] algorithmic bytes, device

    struct Range { int64_t e0, ne; };

    // Pieces per work-stealing chunk: the user's fixed value, else the autotuned one, else 0
    // (sized from the pass's piece total).
    int32_t chunk_for(int L) const {
        if (G->chunk > 0) return G->chunk;
        if (G->tuned_chunk[L] > 0) return G->tuned_chunk[L];
        return 0;
    }

    // Run one pass of the extension kernel over the frontier.
    //   launch 0: batches of at most `batch` embeddings, each sized on the host;
    //   launch 1: one persistent work-stealing launch over the whole frontier (sizes stay on the
    //             device), captured with its prefix kernels into a CUDA graph.  The per-unit piece
    //             prefix takes 8 bytes per (embedding, key position); only when a quarter of the
    //             free device memory cannot hold it is the frontier split into the fewest equal
    //             ranges that fit, each one launch of the same graph;
    //   launch 2: one launch per frontier pattern (the frontier grouped by pattern id), all
    //             captured into one CUDA graph.
    void run_pass(int pass, const LevelSet &in, ExtArgs A, const std::vector<int64_t> &pat_off) {
        const int L = in.L;
        if (in.N == 0) return;
        int64_t B = G->batch > 0 ? G->batch : std::max<int64_t>(1024, ((int64_t)1 << 24) / L);
        std::vector<Range> ranges;
        bool device_total = false;
        if (G->launch == 2 && (int64_t)pat_off.size() == in.P + 1) {  // frontier grouped by pattern
            for (int64_t p = 0; p < in.P; ++p)
                for (int64_t e0 = pat_off[p]; e0 < pat_off[p + 1]; e0 += B)
                    ranges.push_back({e0, std::min(B, pat_off[p + 1] - e0)});
            device_total = true;
        } else if (G->launch == 1) {
            size_t fr = 0, tot = 0;
            ck(cudaMemGetInfo(&fr, &tot), "memory info");
            const int64_t fit = std::max<int64_t>(1 << 20, (int64_t)(fr / 4 / sizeof(int64_t)) / L);   // embeddings
            const int64_t parts = (in.N + fit - 1) / fit;
            const int64_t per = (in.N + parts - 1) / parts;
            for (int64_t e0 = 0; e0 < in.N; e0 += per) ranges.push_back({e0, std::min(per, in.N - e0)});
            device_total = true;
        } else {
            for (int64_t e0 = 0; e0 < in.N; e0 += B) ranges.push_back({e0, std::min(B, in.N - e0)});
        }
        int64_t maxne = 0;
        for (auto &r : ranges) maxne = std::max(maxne, r.ne);
        const int64_t maxu = maxne * L;
        // per-unit piece counts, then their exclusive prefix in place (one extra entry: the total)
        int64_t *base = mem.get<int64_t>(maxu + 1);
        void *tmp = mem.get<char>((int64_t)scan_temp_bytes(maxu) + 16);
        unsigned long long *ctr = mem.get<unsigned long long>(1);
        const int grid = grid_for(L, pass);
        const int64_t warps = (int64_t)grid * 8;
        const bool prof = G->profile != 0;
        A.fv = in.fv;
        A.fpid = in.fpid;
        A.fN = in.N;
        A.unit_base = base;
        A.chunk_ctr = ctr;
        auto launch_ext = [&]() {
            cudaError_t e = pass == PASS_COUNT ? launch_extend_count(L, V, A, grid, st)
                          : pass == PASS_DOMAIN ? launch_extend_domain(L, V, A, grid, st)
                          : pass == PASS_FUSED ? launch_extend_fused(L, A, grid, st)
                                                : launch_extend_emit(L, V, A, grid, st);
            ck(e, "extension kernel");
            rs.launches += 1;
            rs.pass_launches[L][pass] += 1;
        };
        auto bytes = [&](const Range &r) {
            if (prof) ck(launch_unit_bytes(A.g.prow, A.g.ppc, in.fv, in.N, r.e0, r.ne, L, V,
                                           prof_bytes + L * 4 + pass, st), "unit bytes");
        };
        auto new_ev = [&]() {
            ProfEv ev{nullptr, nullptr, L, pass};
            ck(cudaEventCreate(&ev.a), "event");
            ck(cudaEventCreate(&ev.b), "event");
            prof_ev.push_back(ev);
            return prof_ev.size() - 1;
        };
        if (device_total) {
            CapturedGraph cg(st);
            cg.begin();
            for (const Range &r : ranges) {
                ck(launch_unit_counts(A.g, in.fv, in.N, r.e0, r.ne, L, V, A.quota, A.edge_quota, A.qseed, base, st), "unit counts");
                ck(launch_scan_i64(base, base, r.ne * L, tmp, st), "unit scan");
                bytes(r);
                ck(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), st), "memset");
                A.e0 = r.e0;
                A.ne = r.ne;
                A.total = -1;
                A.nchunks = 0;
                A.chunk = chunk_for(L);
                launch_ext();
            }
            cg.end();
            size_t ei = prof ? new_ev() : 0;
            if (prof) ck(cudaEventRecord(prof_ev[ei].a, st), "event record");
            ck(cudaGraphLaunch(cg.exec, st), "graph launch");
            if (prof) ck(cudaEventRecord(prof_ev[ei].b, st), "event record");
        } else {
            for (const Range &r : ranges) {
                ck(launch_unit_counts(A.g, in.fv, in.N, r.e0, r.ne, L, V, A.quota, A.edge_quota, A.qseed, base, st), "unit counts");
                ck(launch_scan_i64(base, base, r.ne * L, tmp, st), "unit scan");
                const int64_t total = d2h(base + r.ne * L, st);
                if (total == 0) continue;
                bytes(r);
                int64_t chunk = chunk_for(L);
                if (chunk <= 0) {   // as the kernel sizes it when the total stays on the device
                    const int64_t per_unit = total / (r.ne * L);
                    chunk = 256;
                    while (chunk < 16384 && total / chunk > warps * 64 && chunk * 2 <= 16 * per_unit) chunk <<= 1;
                }
                A.e0 = r.e0;
                A.ne = r.ne;
                A.total = total;
                A.chunk = (int32_t)chunk;
                A.nchunks = (total + chunk - 1) / chunk;
                ck(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), st), "memset");
                size_t ei = prof ? new_ev() : 0;
                if (prof) ck(cudaEventRecord(prof_ev[ei].a, st), "event record");
                launch_ext();
                if (prof) ck(cudaEventRecord(prof_ev[ei].b, st), "event record");
            }
        }
        mem.release(base);
        mem.release(tmp);
        mem.release(ctr);
    }

    // Frontier grouped by pattern id (launch mode 2): returns host offsets, P+1 entries.
    std::vector<int64_t> group_by_pattern(LevelSet &in) {
        std::vector<int64_t> off;
        // Per-pattern launches need the frontier grouped.  The persistent launch groups it from
        // size 3 on (option "group" = 2): consecutive units then share the pattern, so the count
        // pass's warp tables hit (k = 5 on the 3.7M-vertex graph: count pass -12 %).  Edges keep
        // emission order, whose consecutive units share key vertices (measured faster there).
        const bool grouped = G->launch == 2 || (G->launch == 1 && (G->group == 1 || (G->group == 2 && in.L >= 3)));
        if (!grouped || in.N == 0 || in.P == 0) return off;
        int64_t *cnt = mem.get<int64_t>(in.P);
        int64_t *doff = mem.get<int64_t>(in.P + 1);
        void *tmp = mem.get<char>((int64_t)scan_temp_bytes(in.P) + 16);
        unsigned long long *cur = mem.get<unsigned long long>(in.P);
        ck(launch_u64_to_i64(in.count, cnt, in.P, st), "counts");
        ck(launch_scan_i64(cnt, doff, in.P, tmp, st), "pattern offsets");
        ck(cudaMemsetAsync(cur, 0, sizeof(unsigned long long) * in.P, st), "memset");
        int32_t *nv = mem.get<int32_t>(in.N * in.L);
        int32_t *np = mem.get<int32_t>(in.N);
        ck(launch_group_by_pattern(in.fv, in.fpid, in.N, in.L, doff, cur, nv, np, st), "group by pattern");
        off.resize((size_t)in.P + 1);
        ck(cudaMemcpyAsync(off.data(), doff, sizeof(int64_t) * (in.P + 1), cudaMemcpyDeviceToHost, st), "copy");
        ck(cudaStreamSynchronize(st), "sync");
        if (off[(size_t)in.P] != in.N) fail(FSM_ECUDA, "frontier pattern counts do not add up");
        in.fv = nv;
        in.fpid = np;
        for (void *p : {(void *)cnt, (void *)doff, tmp, (void *)cur}) mem.release(p);
        return off;
    }

    // Autotuner: time a pass on a sample of the frontier for each candidate chunk size and keep
    // the fastest for this level: the domain pass (idempotent: it only ORs domain bits), or, before
    // a one-pass last level, the count pass, whose table the caller wipes afterwards.
    void tune_chunk(const LevelSet &in, ExtArgs A, int pass = PASS_DOMAIN) {
        const int L = in.L;
        if (!G->autotune || G->chunk > 0 || G->tuned_chunk[L] > 0 || in.N == 0) return;
        const int64_t ne = std::min<int64_t>(in.N, std::max<int64_t>(1024, in.N / 32));
        const int64_t nu = ne * L;
        int64_t *cnt = mem.get<int64_t>(nu);
        int64_t *base = mem.get<int64_t>(nu + 1);
        void *tmp = mem.get<char>((int64_t)scan_temp_bytes(nu) + 16);
        unsigned long long *ctr = mem.get<unsigned long long>(1);
        ck(launch_unit_counts(A.g, in.fv, in.N, 0, ne, L, V, A.quota, A.edge_quota, A.qseed, cnt, st), "unit counts");
        ck(launch_scan_i64(cnt, base, nu, tmp, st), "unit scan");
        const int64_t total = d2h(base + nu, st);
        const int grid = grid_for(L, pass);
        A.stats = nullptr;
        A.fv = in.fv;
        A.fpid = in.fpid;
        A.fN = in.N;
        A.e0 = 0;
        A.ne = ne;
        A.unit_base = base;
        A.chunk_ctr = ctr;
        A.total = total;
        cudaEvent_t a, b;
        ck(cudaEventCreate(&a), "event");
        ck(cudaEventCreate(&b), "event");
        float best_ms = 0.f;
        int32_t best = 0;
        for (int32_t chunk : {256, 1024, 4096, 16384}) {
            A.chunk = chunk;
            A.nchunks = (total + chunk - 1) / chunk;
            ck(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), st), "memset");
            ck(cudaEventRecord(a, st), "event record");
            ck(pass == PASS_COUNT ? launch_extend_count(L, V, A, grid, st) : launch_extend_domain(L, V, A, grid, st),
               "extension kernel");
            ck(cudaEventRecord(b, st), "event record");
            ck(cudaEventSynchronize(b), "event sync");
            float ms = 0.f;
            ck(cudaEventElapsedTime(&ms, a, b), "event time");
            rs.launches += 1;
            if (best == 0 || ms < best_ms) { best_ms = ms; best = chunk; }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        G->tuned_chunk[L] = best;
        for (void *p : {(void *)cnt, (void *)base, tmp, (void *)ctr}) mem.release(p);
    }

    int err_word() { return d2h(G->err, st); }

    // Fail with the code a kernel's error word stands for (after the recoverable bits are handled)
    [[noreturn]] void fail_word(int ew) {
        if (ew & FSM_ERR_TIMEOUT)
            fail(FSM_ETIMEOUT, "time limit of " + std::to_string(G->time_limit_ms) + " ms ran out (option time_limit_ms)");
        if (ew & FSM_ERR_BOUNDS) fail(FSM_ECUDA, "a device bounds check failed (error word " + std::to_string(ew) + ")");
        fail(FSM_ECUDA, "extension kernel reported error word " + std::to_string(ew));
    }

    // Extend `in` (size L) to size L+2.  piece_freq == nullptr at the size-3 level.
    // sampled: join only pieces kept by the splitmix64 rule at rate p; every candidate pattern
    // is returned with its sampled support and count and its 32 features.
    LevelSet extend(const LevelSet &in_level, const uint8_t *piece_freq, bool final, bool sampled = false,
                    double p = 1.0, const uint8_t *piece_sel = nullptr) {
        LevelSet in = in_level;
        const std::vector<int64_t> pat_off = group_by_pattern(in);
        const int L = in.L, K = L + (V == FSM_EXPLORE_SV ? 1 : 2);
        LevelSet out;
        out.L = K;
        ExtArgs A;
        memset(&A, 0, sizeof(A));
        A.g = G->dg();
        A.mode = G->mode;
        A.pat_adj = in.adj8;
        A.piece_freq = piece_freq;
        A.piece_sel = piece_sel;
        A.err = G->err;
        A.sampled = sampled ? 1 : 0;
        A.debug = G->debug;
        A.time_limit_ns = (uint64_t)G->time_limit_ms * 1000000ull;
        A.time_start = G->stats + 4;
        if (V == FSM_EXPLORE_TV_QUOTA) {
            // Section 5: size-3 matching (l = 1) draws match_quota candidates per vertex; every
            // join draws join_quota^2 pieces per key group and, joining edges, join_quota edges
            // per key vertex
            A.quota = L == 1 ? G->match_quota : G->join_quota * G->join_quota;
            A.edge_quota = L == 2 ? G->join_quota : 0;
            A.qseed = G->seed;
        }
        if (sampled) {
            // pieces come from the kept directed edges only (rate sqrt(p) each)
            const uint64_t thr = (uint64_t)(std::sqrt(p) * 18446744073709551616.0);
            int64_t *cnt = mem.get<int64_t>(G->n);
            int64_t *prow64 = mem.get<int64_t>(G->n + 1);
            void *tmp = mem.get<char>((int64_t)scan_temp_bytes(G->n) + 16);
            ck(launch_sample_count(A.g, G->seed, thr, cnt, st), "sample count");
            ck(launch_scan_i64(cnt, prow64, G->n, tmp, st), "sample scan");
            const int64_t kept = d2h(prow64 + G->n, st);
            int32_t *prow = mem.get<int32_t>(G->n + 1);
            int32_t *pcol = mem.get<int32_t>(std::max<int64_t>(kept, 1));
            int32_t *pend = mem.get<int32_t>(std::max<int64_t>(kept, 1));
            int64_t *ppc = mem.get<int64_t>(G->n);
            ck(launch_sample_lists(A.g, G->seed, thr, prow64, prow, pcol, pend, ppc, st), "sample lists");
            A.g.prow = prow;
            A.g.pcol = pcol;
            A.g.pend = pend;
            A.g.ppc = ppc;
            A.g.tri_off = nullptr;   // the matrices index the full lists
            A.g.tri_bits = nullptr;
            rs.sampled_edges = kept;
        }
        const int64_t t_live = sampled ? 1 : t;   // sampled counts say nothing about reaching t
        // ---- pass 1: quick patterns and their embedding counts; at the last level (k <= 7, exact
        // mining) also the MNI domains, in the same enumeration, when option "fused" is set
        int64_t cap = G->qp_initial > 0 ? G->qp_initial : (int64_t)1 << 20;
        if (G->qp_initial == 0)
            while (cap < 4 * G->qp_hint[L] && cap < ((int64_t)1 << 30)) cap <<= 1;
        unsigned long long *keys = nullptr, *qcount = nullptr, *used = nullptr, *ptop = nullptr, *ckeys = nullptr,
                           *coff = nullptr;
        long long *soff = nullptr;
        uint32_t *pool = nullptr;
        unsigned long long pool_words = 0;
        bool fused = final && G->fused && V == FSM_EXPLORE_TV && !sampled && K <= 7;
        if (fused) {
            size_t fr = 0, tot = 0;
            ck(cudaMemGetInfo(&fr, &tot), "memory info");
            // twice what the last call needed, else 40% of the free memory
            const unsigned long long cap_words = (unsigned long long)(fr / 4 * 2 / 5);
            pool_words = G->pool_hint[L] ? std::min(cap_words, 2 * G->pool_hint[L] + (1ull << 22)) : cap_words;
            pool_words = std::max<unsigned long long>(pool_words, 1ull << 20);
            if (G->pool_force) pool_words = G->pool_force;
            void *pp = nullptr;
            if (cudaMallocAsync(&pp, pool_words * 4, st) != cudaSuccess) {
                cudaGetLastError();
                fused = false;   // no room for the pool: separate count and domain passes
            } else {
                pool = (uint32_t *)pp;
                mem.ptrs.push_back(pp);
                ptop = mem.get<unsigned long long>(1);
            }
        }
        auto release_pass1 = [&]() {
            for (void *q : {(void *)keys, (void *)qcount, (void *)used, (void *)ckeys, (void *)coff, (void *)soff})
                if (q) mem.release(q);
            keys = qcount = used = ckeys = coff = nullptr;
            soff = nullptr;
        };
        auto clear_pass1 = [&]() {
            ck(launch_fill_u64(keys, FSM_EMPTY_KEY, cap, st), "fill");
            ck(cudaMemsetAsync(qcount, 0, sizeof(unsigned long long) * cap, st), "memset");
            ck(cudaMemsetAsync(used, 0, sizeof(unsigned long long), st), "memset");
            ck(cudaMemsetAsync(G->err, 0, sizeof(int), st), "memset");
            ck(cudaMemsetAsync(G->stats, 0, 3 * sizeof(unsigned long long), st), "memset");
            if (fused) {
                ck(launch_fill_u64(ckeys, FSM_EMPTY_KEY, cap, st), "fill");
                ck(cudaMemsetAsync(coff, 0, sizeof(unsigned long long) * cap, st), "memset");
                ck(cudaMemsetAsync(soff, 0xff, sizeof(long long) * cap * 8, st), "memset");
                ck(cudaMemsetAsync(pool, 0, pool_words * 4, st), "memset");
                ck(cudaMemsetAsync(ptop, 0, sizeof(unsigned long long), st), "memset");
            }
        };
        for (;;) {
            keys = mem.get<unsigned long long>(cap);
            qcount = mem.get<unsigned long long>(cap);
            used = mem.get<unsigned long long>(1);
            if (fused) {
                // the pattern (code) table has as many slots as the quick-pattern table, so it is
                // at most half full whenever that one is
                ckeys = mem.get<unsigned long long>(cap);
                coff = mem.get<unsigned long long>(cap);
                soff = mem.get<long long>(cap * 8);
                A.pat_lab = in.lab8;
                A.code_keys = ckeys;
                A.code_off = coff;
                A.code_mask = (uint64_t)cap - 1;
                A.slot_off = soff;
                A.pool = pool;
                A.pool_top = ptop;
                A.pool_words = pool_words;
                A.cls_size = G->cls_size;
                A.explore = V;
                A.level = L;
            }
            A.qp.keys = keys;
            A.qp.count = qcount;
            A.qp.mask = (uint64_t)cap - 1;
            A.qp.used = used;
            A.qp.max_used = (unsigned long long)(cap / 2);
            A.stats = G->stats;
            clear_pass1();
            if (fused && G->autotune && G->chunk <= 0 && G->tuned_chunk[L] <= 0) {
                // chunk size from trial count passes on a sample; their counts are then wiped
                tune_chunk(in, A, PASS_COUNT);
                clear_pass1();
            }
            run_pass(fused ? PASS_FUSED : PASS_COUNT, in, A, pat_off);
            const int ew = err_word();
            if (ew & (FSM_ERR_TIMEOUT | FSM_ERR_BOUNDS)) fail_word(ew);
            if (ew & FSM_ERR_QP_OVERFLOW) {
                release_pass1();
                if (cap >= ((int64_t)1 << 31)) fail(FSM_EUNSUPPORTED, "more than 2^30 distinct quick patterns in one level");
                cap <<= 2;
                rs.qp_grows += 1;
                continue;
            }
            if (ew & ~(FSM_ERR_POOL | FSM_ERR_CODE_FULL)) fail_word(ew);
            if (ew) {
                // pool or pattern table too small: the one-pass level stopped early; count again
                // in a clean count pass and fill the domains in a domain pass
                fused = false;
                G->pool_hint[L] = 0;
                rs.fused_fallbacks += 1;
                release_pass1();
                continue;
            }
            if (fused) {
                G->pool_hint[L] = d2h(ptop, st);
                rs.fused_pool_words = (int64_t)G->pool_hint[L];
            }
            break;
        }
        unsigned long long st2[3];
        ck(cudaMemcpyAsync(st2, G->stats, sizeof(st2), cudaMemcpyDeviceToHost, st), "copy");
        ck(cudaStreamSynchronize(st), "sync");
        rs.tested += (int64_t)st2[0];
        rs.accepted += (int64_t)st2[1];
        rs.pieces += (int64_t)st2[2];
        rs.pieces_l[L] += (int64_t)st2[2];
        if (final) rs.final_accepted = (int64_t)st2[1];
        // ---- distinct quick patterns -> canonical codes -> pattern ids
        int64_t *slots = mem.get<int64_t>(cap);
        unsigned long long *nq_d = mem.get<unsigned long long>(1);
        ck(cudaMemsetAsync(nq_d, 0, sizeof(unsigned long long), st), "memset");
        ck(launch_qp_compact(keys, cap, slots, nq_d, st), "compact");
        const int64_t nq = (int64_t)d2h(nq_d, st);
        rs.qps += nq;
        G->qp_hint[L] = std::max(G->qp_hint[L], nq);
        int32_t *qpat = mem.get<int32_t>(cap);
        uint64_t *qperm = mem.get<uint64_t>(cap);
        int64_t M = 1;
        while (M < nq) M <<= 1;
        CodeRec *recs = mem.get<CodeRec>(M);
        ck(launch_qp_canon(L, V, keys, slots, nq, in.lab8, in.adj8, recs, qperm, st), "canonicalise");
        ck(launch_sort_codes(recs, nq, st), "sort codes");
        int64_t *flag = mem.get<int64_t>(nq + 1);
        int64_t *ids = mem.get<int64_t>(nq + 1);
        void *stmp = mem.get<char>((int64_t)scan_temp_bytes(nq) + 16);
        unsigned long long *plab = mem.get<unsigned long long>(nq);
        uint64_t *padj = mem.get<uint64_t>(nq);
        ck(launch_assign_patterns(recs, nq, slots, flag, ids, stmp, qpat, plab, padj, st), "assign patterns");
        const int64_t np = nq > 0 ? d2h(ids + nq, st) : 0;
        mem.release(recs);
        // ---- orbits, counts, live patterns, domain bitmaps
        uint64_t *orbit = mem.get<uint64_t>(np);
        int32_t *minorb = mem.get<int32_t>(np);
        unsigned long long *pcount = mem.get<unsigned long long>(np);
        ck(cudaMemsetAsync(pcount, 0, sizeof(unsigned long long) * std::max<int64_t>(np, 1), st), "memset");
        ck(launch_orbits(K, plab, padj, np, orbit, minorb, st), "orbits");
        ck(launch_pattern_counts(slots, nq, qpat, qcount, pcount, st), "pattern counts");
        uint8_t *live = mem.get<uint8_t>(np);
        int64_t *words = mem.get<int64_t>(np * FSM_MAXK);
        int64_t *woff = mem.get<int64_t>(np * FSM_MAXK + 1);
        int64_t *doff = mem.get<int64_t>(np * FSM_MAXK);
        void *stmp2 = mem.get<char>((int64_t)scan_temp_bytes(np * FSM_MAXK) + 16);
        unsigned long long *sigma = mem.get<unsigned long long>(np);
        ck(launch_fill_u64(sigma, ~0ull, np, st), "fill");
        uint32_t *dom = nullptr;
        int64_t *sbase = nullptr;
        rs.patterns = np;
        if (fused) {
            // every pattern has its orbit bitmaps in the pool already: MNI from there
            rs.live = np;
            ck(launch_fused_support(K, plab, padj, orbit, np, ckeys, coff, (uint64_t)cap - 1, G->cls_size, pool, sigma,
                                    st), "fused support");
            if (G->profile) rs.pass_bytes[L][PASS_FUSED] += rs.final_accepted * 4 * K;   // one bitmap word per position
        } else {
            ck(launch_domain_sizes(K, plab, orbit, minorb, pcount, np, t_live, G->cls_size, live, words, st), "domain sizes");
            ck(launch_scan_i64(words, woff, np * FSM_MAXK, stmp2, st), "domain scan");
            ck(launch_domain_offsets(words, woff, np * FSM_MAXK, doff, st), "domain offsets");
            const int64_t nwords = d2h(woff + np * FSM_MAXK, st);
            dom = mem.get<uint32_t>(nwords);
            ck(cudaMemsetAsync(dom, 0, sizeof(uint32_t) * std::max<int64_t>(nwords, 1), st), "memset");
            // live pattern count (for statistics)
            std::vector<uint8_t> hl((size_t)np);
            if (np) {
                ck(cudaMemcpyAsync(hl.data(), live, (size_t)np, cudaMemcpyDeviceToHost, st), "copy");
                ck(cudaStreamSynchronize(st), "sync");
            }
            rs.live = std::count(hl.begin(), hl.end(), (uint8_t)1);
            // ---- pass 2: MNI domains (Definition 2)
            A.qp.pattern = qpat;
            A.qp.perm = qperm;
            A.live = live;
            A.orbit = orbit;
            A.dom_off = doff;
            A.dom = dom;
            sbase = mem.get<int64_t>(cap * FSM_MAXK);
            ck(launch_slot_bases(K, slots, nq, qpat, qperm, live, orbit, doff, sbase, st), "slot bases");
            A.slot_base = sbase;
            A.stats = nullptr;
            if (rs.live > 0) {
                tune_chunk(in, A);
                run_pass(PASS_DOMAIN, in, A, pat_off);
                if (G->profile) {
                    // algorithmic bytes of the domain updates: one 4-byte bitmap word per position
                    // of every accepted join of a live pattern (the list reads are in run_pass)
                    std::vector<unsigned long long> hc((size_t)np);
                    ck(cudaMemcpyAsync(hc.data(), pcount, sizeof(unsigned long long) * np, cudaMemcpyDeviceToHost, st),
                       "copy");
                    ck(cudaStreamSynchronize(st), "sync");
                    int64_t joins = 0;
                    for (int64_t P = 0; P < np; ++P)
                        if (hl[(size_t)P]) joins += (int64_t)hc[(size_t)P];
                    rs.pass_bytes[L][PASS_DOMAIN] += joins * 4 * K;
                }
            }
            ck(launch_support(K, orbit, live, doff, words, dom, np, sigma, st), "support");
        }
        if (pool) {
            mem.release(pool);
            pool = nullptr;
        }
        float *feat = nullptr;
        if (sampled && np > 0) {
            int64_t *aut = mem.get<int64_t>(np);
            feat = mem.get<float>(np * 32);
            ck(launch_aut_size(K, plab, padj, np, aut, st), "automorphisms");
            ck(launch_features(K, plab, padj, orbit, doff, words, dom, pcount, G->cls_size, G->cls_off, G->by_rank,
                               G->row_ptr, G->n, p, t, np, aut, feat, st), "features");
            mem.release(aut);
        }
        int64_t *fflag = mem.get<int64_t>(np + 1);
        int64_t *fscan = mem.get<int64_t>(np + 1);
        int32_t *newid = mem.get<int32_t>(np);
        ck(launch_freq_flags(sigma, np, sampled ? 1 : t, fflag, st), "frequent flags");
        ck(launch_scan_i64(fflag, fscan, np, stmp2, st), "frequent scan");
        ck(launch_new_ids(fflag, fscan, np, newid, st), "new ids");
        const int64_t nf = d2h(fscan + np, st);
        if (dom) mem.release(dom);
        // ---- frequent patterns of size K
        out.P = nf;
        out.lab8 = mem.get<uint64_t>(nf);
        out.adj8 = mem.get<uint64_t>(nf);
        out.clab = mem.get<unsigned long long>(nf);
        out.cadj = mem.get<uint64_t>(nf);
        out.sigma = mem.get<unsigned long long>(nf);
        out.count = mem.get<unsigned long long>(nf);
        ck(launch_gather_frequent(K, newid, np, plab, padj, sigma, pcount, out.clab, out.cadj, out.sigma,
                                  out.count, out.lab8, out.adj8, st), "gather");
        if (feat) {
            // every sampled pattern has a nonzero popcount, so the frequent ids are the identity
            if (nf != np) fail(FSM_ECUDA, "sampled level lost candidate patterns");
            out.feat = feat;
        }
        if (!final && nf > 0) {
            // ---- pass 3: store the frequent size-K embeddings in canonical order
            unsigned long long *sum = mem.get<unsigned long long>(1);
            ck(cudaMemsetAsync(sum, 0, sizeof(unsigned long long), st), "memset");
            ck(launch_sum_frequent(newid, pcount, np, sum, st), "sum");
            const int64_t N2 = (int64_t)d2h(sum, st);
            out.N = N2;
            out.fv = mem.get<int32_t>(N2 * K);
            out.fpid = mem.get<int32_t>(N2);
            unsigned long long *cursor = mem.get<unsigned long long>(1);
            ck(cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), st), "memset");
            A.newid = newid;
            A.out_v = out.fv;
            A.out_pid = out.fpid;
            A.out_N = N2;
            A.out_cursor = cursor;
            run_pass(PASS_EMIT, in, A, pat_off);
            const int64_t wrote = (int64_t)d2h(cursor, st);
            if (wrote != N2) fail(FSM_ECUDA, "frontier emission wrote " + std::to_string(wrote) + " of " + std::to_string(N2));
            if (G->profile) rs.pass_bytes[L][PASS_EMIT] += N2 * 4 * (K + 1);   // output written
            rs.frontier_max = std::max(rs.frontier_max, N2);
            mem.release(sum);
            mem.release(cursor);
        }
        const int ew = err_word();
        if (ew) fail_word(ew);
        if (sbase) mem.release(sbase);
        release_pass1();
        for (void *p : std::initializer_list<void *>{slots, nq_d, qpat, qperm, flag, ids, stmp, plab,
                                                     padj, orbit, minorb, pcount, live, words, woff, doff, stmp2, sigma,
                                                     fflag, fscan, newid})
            mem.release(p);
        rs.levels += 1;
        return out;
    }

    LevelSet level1(bool with_frontier) {
        LevelSet s;
        s.L = 1;
        const int NL = G->NL;
        int32_t *lnew = mem.get<int32_t>(NL);
        s.lab8 = mem.get<uint64_t>(NL);
        s.adj8 = mem.get<uint64_t>(NL);
        s.clab = mem.get<unsigned long long>(NL);
        s.cadj = mem.get<uint64_t>(NL);
        s.sigma = mem.get<unsigned long long>(NL);
        s.count = mem.get<unsigned long long>(NL);
        unsigned long long *nf = mem.get<unsigned long long>(1);
        ck(launch_level1_tables(NL, G->cls_size, t, lnew, s.lab8, s.adj8, s.clab, s.cadj, s.sigma, s.count, nf, st),
           "level 1");
        s.P = (int64_t)d2h(nf, st);
                if (with_frontier) {
            int64_t *flag = mem.get<int64_t>(G->n);
            int64_t *scanned = mem.get<int64_t>(G->n + 1);
            void *tmp = mem.get<char>((int64_t)scan_temp_bytes(G->n) + 16);
            // size: number of vertices with a frequent label
            s.fv = mem.get<int32_t>(G->n);
            s.fpid = mem.get<int32_t>(G->n);
            ck(launch_level1_frontier(G->dg(), lnew, flag, scanned, tmp, s.fv, s.fpid, st), "level 1 frontier");
            s.N = d2h(scanned + G->n, st);
                        mem.release(flag);
            mem.release(scanned);
            mem.release(tmp);
        }
        mem.release(lnew);
        return s;
    }

    LevelSet level2(bool with_frontier) {
        LevelSet s;
        s.L = 2;
        const int NL = G->NL;
        const int64_t NP = (int64_t)NL * NL;
        int64_t *poff = mem.get<int64_t>(NP * 2);
        int64_t *tw = mem.get<int64_t>(1);
        ck(launch_level2_offsets(NL, G->cls_size, poff, tw, st), "level 2 offsets");
        const int64_t words = d2h(tw, st);
        uint32_t *dom = mem.get<uint32_t>(words);
        unsigned long long *pc = mem.get<unsigned long long>(NP);
        unsigned long long *ps = mem.get<unsigned long long>(NP);
        ck(cudaMemsetAsync(dom, 0, sizeof(uint32_t) * std::max<int64_t>(words, 1), st), "memset");
        ck(cudaMemsetAsync(pc, 0, sizeof(unsigned long long) * NP, st), "memset");
        ck(launch_level2_domains(G->dg(), NL, poff, dom, pc, st), "level 2 domains");
        ck(launch_level2_support(NL, G->cls_size, poff, dom, ps, st), "level 2 support");
        int32_t *pnew = mem.get<int32_t>(NP);
        s.lab8 = mem.get<uint64_t>(NP);
        s.adj8 = mem.get<uint64_t>(NP);
        s.clab = mem.get<unsigned long long>(NP);
        s.cadj = mem.get<uint64_t>(NP);
        s.sigma = mem.get<unsigned long long>(NP);
        s.count = mem.get<unsigned long long>(NP);
        unsigned long long *nf = mem.get<unsigned long long>(1);
        ck(launch_level2_tables(NL, ps, pc, t, pnew, s.lab8, s.adj8, s.clab, s.cadj, s.sigma, s.count, nf, st),
           "level 2 tables");
        s.P = (int64_t)d2h(nf, st);
                if (with_frontier && s.P > 0) {
            int64_t *flag = mem.get<int64_t>(G->n);
            int64_t *scanned = mem.get<int64_t>(G->n + 1);
            void *tmp = mem.get<char>((int64_t)scan_temp_bytes(G->n) + 16);
            // stored edges = embeddings of the frequent pairs
            unsigned long long *sum = mem.get<unsigned long long>(1);
            ck(cudaMemsetAsync(sum, 0, sizeof(unsigned long long), st), "memset");
            ck(launch_sum_frequent(pnew, pc, NP, sum, st), "sum");
            s.N = (int64_t)d2h(sum, st);
            mem.release(sum);
            s.fv = mem.get<int32_t>(s.N * 2);
            s.fpid = mem.get<int32_t>(s.N);
            ck(launch_level2_frontier(G->dg(), NL, pnew, flag, scanned, tmp, s.fv, s.N, s.fpid, st), "level 2 frontier");
            const int64_t wrote = d2h(scanned + G->n, st);
            if (wrote != s.N) fail(FSM_ECUDA, "level 2 frontier size mismatch");
                        mem.release(flag);
            mem.release(scanned);
            mem.release(tmp);
        }
        mem.release(poff);
        mem.release(tw);
        mem.release(dom);
        mem.release(pc);
        mem.release(ps);
        mem.release(pnew);
        return s;
    }
};

// Append one pattern's labels and adjacency (both encodings) from its label and adjacency words.
void push_pattern(fsm_result *r, int k, unsigned long long clab, uint64_t code) {
    const int np = k * (k - 1) / 2;
    for (int c = 0; c < k; ++c) r->labels.push_back((int32_t)clab_get(clab, c));
    uint64_t bits = 0, pairs = 0;
    int q = 0;
    for (int i = 0; i < k; ++i)
        for (int j = i + 1; j < k; ++j, ++q)
            if ((code >> (np - 1 - q)) & 1ull) {
                if (k <= 8) bits |= 1ull << (i * k + j);
                pairs |= 1ull << q;
            }
    r->adj.push_back(bits);
    r->pairs.push_back(pairs);
}

void fill_result(fsm_result *r, const LevelSet &s, int k, cudaStream_t st) {
    const int64_t P = s.P;
    std::vector<unsigned long long> lab((size_t)P), sig((size_t)P), cnt((size_t)P);
    std::vector<uint64_t> adj((size_t)P);
    if (P) {
        ck(cudaMemcpyAsync(lab.data(), s.clab, sizeof(unsigned long long) * P, cudaMemcpyDeviceToHost, st), "copy");
        ck(cudaMemcpyAsync(adj.data(), s.cadj, sizeof(uint64_t) * P, cudaMemcpyDeviceToHost, st), "copy");
        ck(cudaMemcpyAsync(sig.data(), s.sigma, sizeof(unsigned long long) * P, cudaMemcpyDeviceToHost, st), "copy");
        ck(cudaMemcpyAsync(cnt.data(), s.count, sizeof(unsigned long long) * P, cudaMemcpyDeviceToHost, st), "copy");
        ck(cudaStreamSynchronize(st), "sync");
    }
    r->k = k;
    r->labels.clear();
    r->adj.clear();
    r->pairs.clear();
    r->support.resize((size_t)P);
    r->count.resize((size_t)P);
    for (int64_t p = 0; p < P; ++p) {
        push_pattern(r, k, lab[p], adj[p]);
        r->support[p] = (int64_t)sig[p];
        r->count[p] = (int64_t)cnt[p];
    }
    r->exact.assign((size_t)P, 1);
}

// Sampled mining, after the sampled last level `cand` (every candidate pattern with its
// smallest sampled orbit popcount in sigma, sampled embedding count, features):
//   option "candidates": return them all with estimates and features;
//   with a model: predict log support; keep predictions >= log t + delta; recount exactly the
//     patterns inside the band with an exact last level restricted to the stored patterns and
//     pieces those patterns can be dissected into; drop the rest;
//   without a model: keep the patterns whose estimate popcount / p reaches t.
void finish_sampled(Miner &m, fsm_result *r, const LevelSet &cand, const LevelSet &stored, const uint8_t *pf,
                    double p, int k) {
    fsm_graph *G = m.G;
    cudaStream_t st = m.st;
    const int64_t P = cand.P;
    std::vector<unsigned long long> lab((size_t)P), sig((size_t)P), cnt((size_t)P);
    std::vector<uint64_t> adj((size_t)P);
    std::vector<float> pred((size_t)P, 0.f), feat;
    std::vector<uint8_t> keep((size_t)P, 0), unc((size_t)P, 0);
    std::vector<int32_t> cls(64, 0);
    ck(cudaMemcpyAsync(cls.data(), G->cls_size, sizeof(int32_t) * 64, cudaMemcpyDeviceToHost, st), "copy");
    if (P) {
        ck(cudaMemcpyAsync(lab.data(), cand.clab, 8 * P, cudaMemcpyDeviceToHost, st), "copy");
        ck(cudaMemcpyAsync(adj.data(), cand.cadj, 8 * P, cudaMemcpyDeviceToHost, st), "copy");
        ck(cudaMemcpyAsync(sig.data(), cand.sigma, 8 * P, cudaMemcpyDeviceToHost, st), "copy");
        ck(cudaMemcpyAsync(cnt.data(), cand.count, 8 * P, cudaMemcpyDeviceToHost, st), "copy");
    }
    // exact results of the recount, by canonical code
    std::map<std::pair<unsigned long long, uint64_t>, std::pair<int64_t, int64_t>> exact;
    const bool use_model = !G->candidates && G->model != nullptr;
    if (G->candidates && P) {
        feat.resize((size_t)P * 32);
        ck(cudaMemcpyAsync(feat.data(), cand.feat, 4 * 32 * P, cudaMemcpyDeviceToHost, st), "copy");
    }
    if (use_model && P) {
        float *dpred = m.mem.get<float>(P);
        uint8_t *dkeep = m.mem.get<uint8_t>(P), *dunc = m.mem.get<uint8_t>(P);
        const int rc = fsm_mlp_predict_device(G->model, cand.feat, P, dpred, st);
        if (rc != FSM_OK) fail(rc, "support prediction failed");
        ck(launch_decide(dpred, P, (float)std::log((double)m.t), (float)G->delta, dkeep, dunc, st), "decide");
        ck(cudaMemcpyAsync(pred.data(), dpred, 4 * P, cudaMemcpyDeviceToHost, st), "copy");
        ck(cudaMemcpyAsync(keep.data(), dkeep, P, cudaMemcpyDeviceToHost, st), "copy");
        ck(cudaMemcpyAsync(unc.data(), dunc, P, cudaMemcpyDeviceToHost, st), "copy");
        ck(cudaStreamSynchronize(st), "sync");
        const int64_t nunc = std::count(unc.begin(), unc.end(), (uint8_t)1);
        m.rs.recount_patterns = nunc;
        if (nunc > 0 && stored.N > 0) {
            // parts the uncertain patterns can be dissected into
            uint8_t *need_s = m.mem.get<uint8_t>(std::max<int64_t>(stored.P, 1));
            uint8_t *need_p = m.mem.get<uint8_t>(FSM_PIECE_SPACE);
            ck(cudaMemsetAsync(need_s, 0, std::max<int64_t>(stored.P, 1), st), "memset");
            ck(cudaMemsetAsync(need_p, 0, FSM_PIECE_SPACE, st), "memset");
            ck(launch_needed_parts(k, cand.clab, cand.cadj, dunc, P, stored.clab, stored.cadj, stored.P, need_s, need_p,
                                   st), "needed parts");
            if (pf) ck(launch_and_u8(need_p, pf, FSM_PIECE_SPACE, st), "and");
            // stored embeddings of the needed patterns only
            int64_t *flag = m.mem.get<int64_t>(stored.N);
            int64_t *scanned = m.mem.get<int64_t>(stored.N + 1);
            void *tmp = m.mem.get<char>((int64_t)scan_temp_bytes(stored.N) + 16);
            ck(launch_flag_count(stored.fpid, stored.N, need_s, flag, st), "flags");
            ck(launch_scan_i64(flag, scanned, stored.N, tmp, st), "scan");
            const int64_t N2 = d2h(scanned + stored.N, st);
            LevelSet sub = stored;
            sub.N = N2;
            sub.fv = m.mem.get<int32_t>(std::max<int64_t>(N2, 1) * stored.L);
            sub.fpid = m.mem.get<int32_t>(std::max<int64_t>(N2, 1));
            ck(launch_compact_frontier(stored.fv, stored.fpid, stored.N, stored.L, need_s, flag, scanned, tmp, sub.fv,
                                       N2, sub.fpid, st), "compact");
            // per-pattern counts of the restricted frontier (needed only by per-pattern launches)
            if (G->launch != 0) {
                unsigned long long *c2 = m.mem.get<unsigned long long>(std::max<int64_t>(stored.P, 1));
                ck(cudaMemsetAsync(c2, 0, 8 * std::max<int64_t>(stored.P, 1), st), "memset");
                ck(launch_keep_counts(stored.count, need_s, stored.P, c2, st), "counts");
                sub.count = c2;
            }
            m.rs.recount_frontier = N2;
            LevelSet ex = m.extend(sub, pf, true, false, 1.0, need_p);
            std::vector<unsigned long long> el((size_t)ex.P), es((size_t)ex.P), ec((size_t)ex.P);
            std::vector<uint64_t> ea((size_t)ex.P);
            if (ex.P) {
                ck(cudaMemcpyAsync(el.data(), ex.clab, 8 * ex.P, cudaMemcpyDeviceToHost, st), "copy");
                ck(cudaMemcpyAsync(ea.data(), ex.cadj, 8 * ex.P, cudaMemcpyDeviceToHost, st), "copy");
                ck(cudaMemcpyAsync(es.data(), ex.sigma, 8 * ex.P, cudaMemcpyDeviceToHost, st), "copy");
                ck(cudaMemcpyAsync(ec.data(), ex.count, 8 * ex.P, cudaMemcpyDeviceToHost, st), "copy");
            }
            ck(cudaStreamSynchronize(st), "sync");
            for (int64_t q = 0; q < ex.P; ++q) exact[{el[q], ea[q]}] = {(int64_t)es[q], (int64_t)ec[q]};
        }
    }
    ck(cudaStreamSynchronize(st), "sync");
    r->k = k;
    for (int64_t q = 0; q < P; ++q) {
        const double est = (double)sig[q] / p;
        int64_t sup = 0, c = 0;
        int32_t ex = 0;
        if (G->candidates) {
            sup = (int64_t)std::llround(est);
            c = (int64_t)std::llround((double)cnt[q] / p);
        } else if (use_model) {
            if (keep[q]) {
                // predicted support, clamped to what is certain: the sampled domains are subsets
                // of the true ones (lower bound) and no orbit outgrows its label class (upper)
                double hi = 1e300;
                for (int cc = 0; cc < k; ++cc)
                    hi = std::min(hi, (double)cls[clab_get(lab[q], cc)]);
                const double lo = (double)sig[q];
                const double pr = std::exp(std::min((double)pred[q], 60.0));
                sup = (int64_t)std::llround(std::max(lo, std::min(hi, pr)));
                c = (int64_t)std::llround((double)cnt[q] / p);
            } else if (unc[q]) {
                auto it = exact.find({lab[q], adj[q]});
                if (it == exact.end()) continue;   // recounted below t
                sup = it->second.first;
                c = it->second.second;
                ex = 1;
            } else {
                continue;
            }
        } else {
            if (est < (double)m.t) continue;
            sup = (int64_t)std::llround(est);
            c = (int64_t)std::llround((double)cnt[q] / p);
        }
        push_pattern(r, k, lab[q], adj[q]);
        r->support.push_back(sup);
        r->count.push_back(c);
        r->exact.push_back(ex);
        if (G->candidates) r->features.insert(r->features.end(), feat.begin() + q * 32, feat.begin() + q * 32 + 32);
    }
    m.rs.candidates_sampled = P;
}

} // namespace

// ============================================================================ C ABI

extern "C" {

const char *fsm_last_error(void) { return g_last_error.c_str(); }

int fsm_load_graph(const int32_t *row_ptr, const int32_t *col, const int32_t *labels, int32_t n,
                   int32_t num_labels, fsm_graph **out) {
    fsm_graph *g = nullptr;
    try {
        if (!out) fail(FSM_EINVAL, "out is NULL");
        *out = nullptr;
        if (!row_ptr || !labels || n < 1) fail(FSM_EINVAL, "row_ptr/labels must be non-NULL and n >= 1");
        if (num_labels < 1 || num_labels > 64) fail(FSM_EINVAL, "num_labels must be in [1, 64]");
        if (row_ptr[0] != 0) fail(FSM_EINVAL, "row_ptr[0] must be 0");
        for (int32_t v = 0; v < n; ++v)
            if (row_ptr[v + 1] < row_ptr[v]) fail(FSM_EINVAL, "row_ptr must be nondecreasing");
        const int64_t nnz = row_ptr[n];
        if (nnz > 0 && !col) fail(FSM_EINVAL, "col is NULL");
        if (nnz >= ((int64_t)1 << 31) - 1) fail(FSM_EUNSUPPORTED, "nnz must be below 2^31 - 1");
        g = new fsm_graph();
        ck(cudaGetDevice(&g->device), "cudaGetDevice");
        keep_pool(g->device);
        ck(cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device), "device attribute");
        ck(cudaStreamCreateWithFlags(&g->own_stream, cudaStreamNonBlocking), "stream create");
        g->stream = g->own_stream;
        g->n = n;
        g->NL = num_labels;
        g->nnz = nnz;
        cudaStream_t st = g->stream;
        auto dalloc = [&](void **p, size_t bytes) { ck(cudaMallocAsync(p, std::max<size_t>(bytes, 16), st), "device allocation"); };
        dalloc((void **)&g->row_ptr, sizeof(int32_t) * (n + 1));
        dalloc((void **)&g->col, sizeof(int32_t) * nnz);
        dalloc((void **)&g->labels, sizeof(int32_t) * n);
        dalloc((void **)&g->rank, sizeof(int32_t) * n);
        dalloc((void **)&g->cls_size, sizeof(int32_t) * 64);
        dalloc((void **)&g->end_off, sizeof(int32_t) * nnz);
        dalloc((void **)&g->piece_cnt, sizeof(int64_t) * n);
        dalloc((void **)&g->err, sizeof(int) * 4);
        dalloc((void **)&g->stats, sizeof(unsigned long long) * 8);
        ck(cudaMemcpyAsync(g->row_ptr, row_ptr, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st), "copy");
        if (nnz) ck(cudaMemcpyAsync(g->col, col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st), "copy");
        ck(cudaMemcpyAsync(g->labels, labels, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st), "copy");
        ck(cudaMemsetAsync(g->err, 0, sizeof(int) * 4, st), "memset");
        ck(cudaMemsetAsync(g->cls_size, 0, sizeof(int32_t) * 64, st), "memset");
        ck(launch_validate(g->dg(), num_labels, g->err, st), "validate");
        const int ew = d2h(g->err, st);
        if (ew) fail(FSM_EINVAL, "malformed CSR: rows must be sorted, symmetric, without self-loops or duplicates, labels in range");
        ck(launch_prepare(g->dg(), g->piece_cnt, g->end_off, g->rank, g->cls_size, st), "prepare");
        {
            // Neighbour-adjacency matrices for the triangle test of centre pairs, for vertices
            // of degree >= dmin; dmin doubles until they fit the budget.
            int64_t *words = nullptr, *off = nullptr;
            void *tmp = nullptr;
            dalloc((void **)&words, sizeof(int64_t) * std::max<int64_t>(n, 1));
            dalloc((void **)&off, sizeof(int64_t) * (n + 1));
            dalloc(&tmp, scan_temp_bytes(n) + 16);
            int32_t dmin = FSM_TRI_DMIN;
            int64_t total = 0;
            for (;;) {
                ck(launch_tri_words(g->dg(), dmin, words, st), "matrix sizes");
                ck(launch_scan_i64(words, off, n, tmp, st), "matrix offsets");
                total = d2h(off + n, st);
                if (total * 4 <= FSM_TRI_BUDGET || dmin > (1 << 30) / 2) break;
                dmin *= 2;
            }
            if (total * 4 > FSM_TRI_BUDGET) total = 0, dmin = 0x7fffffff;
            dalloc((void **)&g->tri_off, sizeof(int64_t) * std::max<int64_t>(n, 1));
            dalloc((void **)&g->tri_bits, sizeof(uint32_t) * std::max<int64_t>(total, 1));
            ck(cudaMemsetAsync(g->tri_bits, 0, sizeof(uint32_t) * std::max<int64_t>(total, 1), st), "memset");
            ck(launch_tri_bits(g->dg(), dmin, off, g->tri_off, g->tri_bits, st), "neighbour matrices");
            cudaFreeAsync(words, st);
            cudaFreeAsync(off, st);
            cudaFreeAsync(tmp, st);
        }
        dalloc((void **)&g->by_rank, sizeof(int32_t) * n);
        dalloc((void **)&g->cls_off, sizeof(int64_t) * 65);
        ck(launch_by_rank(g->dg(), num_labels, g->cls_size, g->cls_off, g->by_rank, st), "rank table");
        ck(cudaStreamSynchronize(st), "sync");
        *out = g;
        return FSM_OK;
    } catch (const FsmError &e) {
        if (g) fsm_free_graph(g);
        return set_error(e);
    }
}

int fsm_set_option(fsm_graph *g, const char *key, int64_t value) {
    try {
        if (!g || !key) fail(FSM_EINVAL, "graph and key must be non-NULL");
        std::string k(key);
        if (k == "mode") {
            if (value != 0 && value != 1) fail(FSM_EINVAL, "mode must be 0 (edge-induced) or 1 (vertex-induced)");
            g->mode = (int)value;
        } else if (k == "stream") {
            g->stream = value ? (cudaStream_t)(intptr_t)value : g->own_stream;
        } else if (k == "fused") {
            if (value != 0 && value != 1) fail(FSM_EINVAL, "fused must be 0 or 1");
            g->fused = (int)value;
        } else if (k == "fused_pool") {
            if (value < 0) fail(FSM_EINVAL, "fused_pool must be >= 0");
            g->pool_force = (unsigned long long)value;
        } else if (k == "seed") {
            g->seed = (uint64_t)value;
        } else if (k == "candidates") {
            if (value != 0 && value != 1) fail(FSM_EINVAL, "candidates must be 0 or 1");
            g->candidates = (int)value;
        } else if (k == "model") {
            g->model = (const fsm_mlp *)(intptr_t)value;
        } else if (k == "delta_milli") {
            if (value < 0 || value > 20000) fail(FSM_EINVAL, "delta_milli must be in [0, 20000]");
            g->delta = (double)value / 1000.0;
        } else if (k == "profile") {
            if (value != 0 && value != 1) fail(FSM_EINVAL, "profile must be 0 or 1");
            g->profile = (int)value;
        } else if (k == "launch") {
            if (value < 0 || value > 2) fail(FSM_EINVAL, "launch must be 0, 1 or 2");
            g->launch = (int)value;
        } else if (k == "group") {
            if (value < 0 || value > 2) fail(FSM_EINVAL, "group must be 0, 1 or 2");
            g->group = (int)value;
        } else if (k == "autotune") {
            if (value != 0 && value != 1) fail(FSM_EINVAL, "autotune must be 0 or 1");
            g->autotune = (int)value;
            if (!value)
                for (auto &c : g->tuned_chunk) c = 0;
        } else if (k == "chunk") {
            if (value != 0 && (value < 32 || value > 65536 || (value & (value - 1)))) fail(FSM_EINVAL, "chunk must be 0 or a power of two in [32, 65536]");
            g->chunk = (int32_t)value;
        } else if (k == "debug") {
            if (value != 0 && value != 1) fail(FSM_EINVAL, "debug must be 0 or 1");
            g->debug = (int)value;
        } else if (k == "time_limit_ms") {
            if (value < 0) fail(FSM_EINVAL, "time_limit_ms must be >= 0");
            g->time_limit_ms = value;
        } else if (k == "fail_alloc_after") {
            if (value < 0) fail(FSM_EINVAL, "fail_alloc_after must be >= 0");
            g->fail_alloc_after = value;
        } else if (k == "join_quota") {
            if (value < 0 || value > 65536) fail(FSM_EINVAL, "join_quota must be in [0, 65536]");
            g->join_quota = value;
        } else if (k == "match_quota") {
            if (value < 0 || value > ((int64_t)1 << 32)) fail(FSM_EINVAL, "match_quota must be in [0, 2^32]");
            g->match_quota = value;
        } else if (k == "explore") {
            if (value != 0 && value != 1) fail(FSM_EINVAL, "explore must be 0 (two-vertex) or 1 (single-vertex)");
            g->explore = (int)value;
        } else if (k == "quick_pattern") {
            if (value != 0 && value != 1) fail(FSM_EINVAL, "quick_pattern must be 0 (index-based) or 1 (edge list)");
            g->quick_pattern = (int)value;
        } else if (k == "qp_capacity") {
            if (value != 0 && (value < 64 || value > ((int64_t)1 << 30) || (value & (value - 1))))
                fail(FSM_EINVAL, "qp_capacity must be 0 or a power of two in [64, 2^30]");
            g->qp_initial = value;
        } else if (k == "batch") {
            if (value != 0 && value < 1024) fail(FSM_EINVAL, "batch must be 0 or >= 1024");
            g->batch = value;
        } else {
            fail(FSM_EINVAL, "unknown option '" + k + "'");
        }
        return FSM_OK;
    } catch (const FsmError &e) {
        return set_error(e);
    }
}

int fsm_mine(fsm_graph *g, int32_t k, int64_t min_support, double sample_rate, fsm_result **out) {
    fsm_result *r = nullptr;
    try {
        if (!out) fail(FSM_EINVAL, "out is NULL");
        *out = nullptr;
        if (!g) fail(FSM_EINVAL, "graph is NULL");
        if (k < 1 || k > FSM_MAXK) fail(FSM_EINVAL, "k must be in [1, 9]");
        if (min_support < 1) fail(FSM_EINVAL, "min_support must be >= 1");
        if (!(sample_rate > 0.0 && sample_rate <= 1.0)) fail(FSM_EINVAL, "sample_rate must be in (0, 1]");
        const bool sampled = sample_rate < 1.0 && k >= 3;   // levels 1 and 2 join no pieces
        const bool quota = g->join_quota > 0 || g->match_quota > 0;
        const int V = g->explore == 1 ? FSM_EXPLORE_SV : g->quick_pattern == 1 ? FSM_EXPLORE_TV_EDGELIST
                    : quota ? FSM_EXPLORE_TV_QUOTA : FSM_EXPLORE_TV;
        if (g->explore + g->quick_pattern + (quota ? 1 : 0) > 1)
            fail(FSM_EUNSUPPORTED, "single-vertex exploration, edge-list quick patterns and sampling quotas exclude each other");
        if (V != FSM_EXPLORE_TV && sampled)
            fail(FSM_EUNSUPPORTED, "rate-sampled mining runs with two-vertex exploration and index-based quick patterns, "
                                   "without sampling quotas, only");
        if ((V == FSM_EXPLORE_SV || V == FSM_EXPLORE_TV_EDGELIST) && k > 7)
            fail(FSM_EUNSUPPORTED, "the exploration ablations support k <= 7");
        if (sampled && k > 8)
            fail(FSM_EUNSUPPORTED, "rate-sampled mining (32 features over at most 8 positions) supports k <= 8");
        ck(cudaSetDevice(g->device), "cudaSetDevice");
        cudaStream_t st = g->stream;
        cudaEvent_t ev0, ev1, evf;
        ck(cudaEventCreate(&ev0), "event");
        ck(cudaEventCreate(&ev1), "event");
        ck(cudaEventCreate(&evf), "event");
        const int64_t l0 = launches_so_far();
        ck(cudaEventRecord(ev0, st), "event record");
        RunStats rs;
        r = new fsm_result();
        {
            Arena mem(st);
            mem.fail_at = g->fail_alloc_after;
            ck(launch_stamp_time(g->stats + 4, st), "time stamp");
            Miner m{g, st, mem, min_support, rs};
            m.V = V;
            if (g->profile) {
                m.prof_bytes = mem.get<unsigned long long>((FSM_MAXL + 1) * 4);
                ck(cudaMemsetAsync(m.prof_bytes, 0, sizeof(unsigned long long) * (FSM_MAXL + 1) * 4, st), "memset");
            }
            LevelSet res;
            if (k == 1) {
                res = m.level1(false);
                ck(cudaEventRecord(evf, st), "event record");
            } else if (V == FSM_EXPLORE_SV) {
                // single-vertex exploration: levels 1 -> 2 -> ... -> k, no size-3 pruning table
                LevelSet cur = m.level1(true);
                while (cur.L < k) {
                    const bool fin = cur.L + 1 == k;
                    if (fin) ck(cudaEventRecord(evf, st), "event record");
                    cur = m.extend(cur, nullptr, fin);
                }
                res = cur;
            } else if (k == 2) {
                res = m.level2(false);
                ck(cudaEventRecord(evf, st), "event record");
            } else {
                LevelSet s1 = m.level1(true);
                const bool odd = (k & 1) != 0;
                LevelSet stored = s1;            // the level the last one extends
                const uint8_t *pf = nullptr;
                if (k == 3) {
                    ck(cudaEventRecord(evf, st), "event record");
                    res = m.extend(s1, nullptr, true, sampled, sample_rate);
                } else {
                    LevelSet s3 = m.extend(s1, nullptr, !odd);
                    uint8_t *pfm = mem.get<uint8_t>(FSM_PIECE_SPACE);
                    ck(cudaMemsetAsync(pfm, 0, FSM_PIECE_SPACE, st), "memset");
                    ck(launch_piece_table(s3.clab, s3.cadj, s3.P, pfm, st), "piece table");
                    pf = pfm;
                    LevelSet cur = odd ? s3 : m.level2(true);
                    while (cur.L + 2 <= k) {
                        const bool fin = cur.L + 2 == k;
                        if (fin) {
                            ck(cudaEventRecord(evf, st), "event record");
                            stored = cur;
                        }
                        cur = m.extend(cur, pf, fin, fin && sampled, sample_rate);
                    }
                    res = cur;
                }
                if (sampled) {
                    ck(cudaEventRecord(ev1, st), "event record");
                    finish_sampled(m, r, res, stored, pf, sample_rate, k);
                    res.P = -1;   // result already filled
                }
            }
            if (res.P >= 0) {
                ck(cudaEventRecord(ev1, st), "event record");
                fill_result(r, res, k, st);
                // sampling quotas: supports and counts are those of the drawn embeddings (lower
                // bounds of the exact ones)
                if (V == FSM_EXPLORE_TV_QUOTA) r->exact.assign(r->exact.size(), 0);
            }
            if (g->profile) {
                unsigned long long pb[(FSM_MAXL + 1) * 4];
                ck(cudaMemcpyAsync(pb, m.prof_bytes, sizeof(pb), cudaMemcpyDeviceToHost, st), "copy");
                ck(cudaStreamSynchronize(st), "sync");
                for (int L = 0; L <= FSM_MAXL; ++L)
                    for (int p = 0; p < 4; ++p) rs.pass_bytes[L][p] += (int64_t)pb[L * 4 + p];
                for (auto &ev : m.prof_ev) {
                    float ems = 0.f;
                    ck(cudaEventElapsedTime(&ems, ev.a, ev.b), "event time");
                    rs.pass_ns[ev.L][ev.pass] += (double)ems * 1e6;
                }
            }
            for (auto &ev : m.prof_ev) {
                cudaEventDestroy(ev.a);
                cudaEventDestroy(ev.b);
            }
        }
        ck(cudaStreamSynchronize(st), "sync");
        float ms = 0.f, fms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventElapsedTime(&fms, evf, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        cudaEventDestroy(evf);
        r->stats["k"] = k;
        r->stats["levels"] = rs.levels;
        r->stats["candidates"] = rs.tested;
        r->stats["pieces"] = rs.pieces;
        r->stats["embeddings"] = rs.accepted;
        r->stats["final_embeddings"] = rs.final_accepted;
        r->stats["quick_patterns"] = rs.qps;
        r->stats["patterns"] = rs.patterns;
        r->stats["live_patterns"] = rs.live;
        r->stats["frontier_max"] = rs.frontier_max;
        r->stats["kernel_launches"] = (launches_so_far() - l0) + rs.launches;
        r->stats["time_ns"] = (int64_t)((double)ms * 1e6);
        r->stats["final_level_ns"] = (int64_t)((double)fms * 1e6);
        r->stats["sampled_candidates"] = rs.candidates_sampled;
        r->stats["recount_patterns"] = rs.recount_patterns;
        r->stats["recount_frontier"] = rs.recount_frontier;
        r->stats["sampled_edges"] = rs.sampled_edges;
        r->stats["qp_grows"] = rs.qp_grows;
        r->stats["fused_fallbacks"] = rs.fused_fallbacks;
        r->stats["fused_pool_words"] = rs.fused_pool_words;
        for (int L = 1; L <= FSM_MAXL; ++L) r->stats["chunk_l" + std::to_string(L)] = g->tuned_chunk[L];
        for (int L = 1; L <= FSM_MAXL; ++L) r->stats["pieces_l" + std::to_string(L)] = rs.pieces_l[L];
        const char *pn[4] = {"count", "domain", "emit", "fused"};
        for (int p = 0; p < 4; ++p) {
            double ns = 0;
            int64_t nl = 0, nb = 0;
            for (int L = 1; L <= FSM_MAXL; ++L) {
                const std::string sfx = "_l" + std::to_string(L);
                r->stats[std::string(pn[p]) + "_ns" + sfx] = (int64_t)rs.pass_ns[L][p];
                r->stats[std::string(pn[p]) + "_launches" + sfx] = rs.pass_launches[L][p];
                r->stats[std::string(pn[p]) + "_bytes" + sfx] = rs.pass_bytes[L][p];
                ns += rs.pass_ns[L][p];
                nl += rs.pass_launches[L][p];
                nb += rs.pass_bytes[L][p];
            }
            r->stats[std::string(pn[p]) + "_ns"] = (int64_t)ns;
            r->stats[std::string(pn[p]) + "_launches"] = nl;
            r->stats[std::string(pn[p]) + "_bytes"] = nb;
        }
        *out = r;
        return FSM_OK;
    } catch (const FsmError &e) {
        delete r;
        return set_error(e);
    }
}

int64_t fsm_result_count(const fsm_result *r) {
    if (!r) { g_last_error = "result is NULL"; return FSM_EINVAL; }
    return (int64_t)r->support.size();
}

int fsm_result_get(const fsm_result *r, int64_t i, int32_t *labels_k, uint64_t *adj_bits, int64_t *support) {
    if (!r || i < 0 || i >= (int64_t)r->support.size()) { g_last_error = "bad result or index"; return FSM_EINVAL; }
    if (adj_bits && r->k > 8) { g_last_error = "adj_bits holds k <= 8: use fsm_result_pairs"; return FSM_EUNSUPPORTED; }
    if (labels_k) std::memcpy(labels_k, r->labels.data() + (size_t)i * r->k, sizeof(int32_t) * r->k);
    if (adj_bits) *adj_bits = r->adj[(size_t)i];
    if (support) *support = r->support[(size_t)i];
    return FSM_OK;
}

int fsm_result_embeddings(const fsm_result *r, int64_t i, int64_t *count) {
    if (!r || !count || i < 0 || i >= (int64_t)r->count.size()) { g_last_error = "bad result or index"; return FSM_EINVAL; }
    *count = r->count[(size_t)i];
    return FSM_OK;
}

int fsm_result_copy(const fsm_result *r, int32_t *labels, uint64_t *adj_bits, int64_t *support, int64_t *embeddings) {
    if (!r) { g_last_error = "result is NULL"; return FSM_EINVAL; }
    if (adj_bits && r->k > 8) { g_last_error = "adj_bits holds k <= 8: use fsm_result_pairs"; return FSM_EUNSUPPORTED; }
    const size_t P = r->support.size();
    if (labels && P) std::memcpy(labels, r->labels.data(), sizeof(int32_t) * P * r->k);
    if (adj_bits && P) std::memcpy(adj_bits, r->adj.data(), sizeof(uint64_t) * P);
    if (support && P) std::memcpy(support, r->support.data(), sizeof(int64_t) * P);
    if (embeddings && P) std::memcpy(embeddings, r->count.data(), sizeof(int64_t) * P);
    return FSM_OK;
}

int fsm_result_pairs(const fsm_result *r, uint64_t *pairs) {
    if (!r || !pairs) { g_last_error = "NULL argument"; return FSM_EINVAL; }
    if (!r->pairs.empty()) std::memcpy(pairs, r->pairs.data(), sizeof(uint64_t) * r->pairs.size());
    return FSM_OK;
}

int fsm_result_exact(const fsm_result *r, int32_t *exact) {
    if (!r || !exact) { g_last_error = "NULL argument"; return FSM_EINVAL; }
    if (!r->exact.empty()) std::memcpy(exact, r->exact.data(), sizeof(int32_t) * r->exact.size());
    return FSM_OK;
}

int fsm_result_features(const fsm_result *r, float *features) {
    if (!r || !features) { g_last_error = "NULL argument"; return FSM_EINVAL; }
    if (r->features.size() != r->support.size() * 32) {
        g_last_error = "no features: mine with sample_rate < 1 and option candidates = 1";
        return FSM_EINVAL;
    }
    if (!r->features.empty()) std::memcpy(features, r->features.data(), sizeof(float) * r->features.size());
    return FSM_OK;
}

int fsm_result_stat(const fsm_result *r, const char *key, int64_t *value) {
    if (!r || !key || !value) { g_last_error = "NULL argument"; return FSM_EINVAL; }
    auto it = r->stats.find(key);
    if (it == r->stats.end()) { g_last_error = std::string("unknown stat '") + key + "'"; return FSM_EINVAL; }
    *value = it->second;
    return FSM_OK;
}

void fsm_free_result(fsm_result *r) { delete r; }

void fsm_free_graph(fsm_graph *g) {
    if (!g) return;
    cudaStream_t st = g->stream ? g->stream : g->own_stream;
    void *ps[] = {g->row_ptr, g->col, g->labels, g->rank, g->cls_size, g->end_off, g->piece_cnt, g->tri_off, g->tri_bits, g->err, g->stats,
                  g->by_rank, g->cls_off};
    for (void *p : ps)
        if (p) cudaFreeAsync(p, st);
    if (st) cudaStreamSynchronize(st);
    if (g->own_stream) cudaStreamDestroy(g->own_stream);
    delete g;
}

int fsm_debug_dissect(int32_t k, const int32_t *ids, const uint32_t *adj, uint32_t *l_mask, int32_t *join,
                      int32_t *used_fallback) {
    if (k < 3 || k > FSM_MAXK || !ids || !adj || !l_mask || !join || !used_fallback) {
        g_last_error = "k must be in [3, 8] and pointers non-NULL";
        return FSM_EINVAL;
    }
    const uint32_t all = (1u << k) - 1u;
    for (int i = 0; i < k; ++i) {
        if ((adj[i] & ~all) || (adj[i] >> i & 1u)) { g_last_error = "adjacency out of range or self-loop"; return FSM_EINVAL; }
        for (int j = 0; j < k; ++j)
            if (((adj[i] >> j) & 1u) != ((adj[j] >> i) & 1u)) { g_last_error = "adjacency not symmetric"; return FSM_EINVAL; }
        for (int j = i + 1; j < k; ++j)
            if (ids[i] == ids[j]) { g_last_error = "ids not distinct"; return FSM_EINVAL; }
    }
    if (!mask_connected(all, adj, k)) { g_last_error = "graph not connected"; return FSM_EINVAL; }
    uint32_t lm = 0;
    int jn = -1;
    const bool greedy = dissect3(k, ids, adj, lm, jn);
    if (lm == 0) { g_last_error = "no dissection exists"; return FSM_EINVAL; }
    *l_mask = lm;
    *join = jn;
    *used_fallback = greedy ? 0 : 1;
    return FSM_OK;
}

} // extern "C"
