// fsm_noalloc.cu -- MNI supports of every labeled edge pattern without any device allocation.
//
// Some callers cannot call cudaMalloc: code running inside an allocator's own callback, a
// process whose device memory is fully reserved by another framework's pool, or a host that
// must not let a library grow its device footprint after start-up.  fsm_edge_supports_noalloc
// serves them.  It runs the same size-2 computation as fsm_mine(k = 2): label classes, a rank
// per vertex inside its class, one domain bitmap per label-pair orbit, popcounts.  All of its
// scratch lives in one file-scope static device array of FSM_NOALLOC_SCRATCH_BYTES.  The
// array is reserved when the library's device code is loaded on a GPU and stays there until
// the process exits.
#include "fsm.h"
#include "fsm_kernels.cuh"

#include <algorithm>
#include <mutex>
#include <string>

namespace fsm {
void set_last_error_message(const std::string &m);   // defined with the rest of the C ABI
}

#define FSM_NOALLOC_SCRATCH_WORDS (16u * 1024u * 1024u)   // 64 MiB of 32-bit words

static __device__ __align__(256) uint32_t g_noalloc_scratch[FSM_NOALLOC_SCRATCH_WORDS];

namespace {

std::mutex g_noalloc_mu;
uint32_t *g_noalloc_ptr[64] = {};   // device address of g_noalloc_scratch, per device

__global__ void noalloc_rank_kernel(const int32_t *labels, int32_t n, int32_t *rank, int32_t *cls_size) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        rank[v] = atomicAdd(cls_size + labels[v], 1);
}

// word offsets inside the scratch array (each region 256-byte aligned)
struct Layout {
    uint64_t cls, err, total, pair_count, pair_off, rank, dom, end;
};

uint64_t align64(uint64_t w) { return (w + 63u) & ~(uint64_t)63u; }

Layout layout(int32_t n, int32_t NL) {
    Layout L;
    const uint64_t np = (uint64_t)NL * (uint64_t)NL;
    L.cls = 0;                                   // int32[64]
    L.err = align64(L.cls + 64);                 // int32[4]
    L.total = align64(L.err + 4);                // int64[1]
    L.pair_count = align64(L.total + 2);         // uint64[NL*NL]
    L.pair_off = align64(L.pair_count + 2 * np); // int64[NL*NL*2]
    L.rank = align64(L.pair_off + 4 * np);       // int32[n]
    L.dom = align64(L.rank + (uint64_t)n);
    // every label class appears in NL label-pair orbits, so the bitmaps need at most
    // NL * sum_l ceil(|V_l| / 32) <= NL * (ceil(n / 32) + NL) words
    L.end = L.dom + (uint64_t)NL * (((uint64_t)n + 31u) / 32u + (uint64_t)NL);
    return L;
}

} // namespace

extern "C" int fsm_edge_supports_noalloc(const int32_t *d_row_ptr, const int32_t *d_col, const int32_t *d_labels,
                                         int32_t n, int32_t num_labels, uint64_t *d_support, uint64_t *d_count,
                                         void *stream) {
    auto err = [](int code, const std::string &m) {
        fsm::set_last_error_message(m);
        return code;
    };
    if (!d_row_ptr || !d_labels || !d_support || !d_count || n < 1)
        return err(FSM_EINVAL, "d_row_ptr, d_labels, d_support, d_count must be non-NULL and n >= 1");
    if (num_labels < 1 || num_labels > 64) return err(FSM_EINVAL, "num_labels must be in [1, 64]");
    const Layout L = layout(n, num_labels);
    if (L.end > FSM_NOALLOC_SCRATCH_WORDS)
        return err(FSM_EUNSUPPORTED,
                   "graph too large for the fixed scratch of fsm_edge_supports_noalloc: needs " +
                       std::to_string(L.end * 4) + " bytes, the static array holds " +
                       std::to_string((uint64_t)FSM_NOALLOC_SCRATCH_WORDS * 4) + " bytes");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return err(FSM_ECUDA, "no current CUDA device");
    uint32_t *base = nullptr;
    {
        // set-up, once per device with that device current: the host-side name of the array is
        // only a stand-in, so its device address is looked up and cached
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return err(FSM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_noalloc_ptr[dev] = (uint32_t *)p;
        }
        base = g_noalloc_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *cls = (int32_t *)(base + L.cls);
    int *errw = (int *)(base + L.err);
    int64_t *total = (int64_t *)(base + L.total);
    unsigned long long *pair_count = (unsigned long long *)(base + L.pair_count);
    int64_t *pair_off = (int64_t *)(base + L.pair_off);
    int32_t *rank = (int32_t *)(base + L.rank);
    uint32_t *dom = base + L.dom;
    int32_t nnz = 0;
    // the whole used region starts at zero: the array keeps the previous call's contents
    cudaError_t e = cudaMemsetAsync(base, 0, L.end * sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nnz, d_row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return err(FSM_ECUDA, std::string("set-up copy: ") + cudaGetErrorString(e));
    if (nnz < 0) return err(FSM_EINVAL, "row_ptr[n] is negative");
    if (nnz > 0 && !d_col) return err(FSM_EINVAL, "d_col is NULL");
    fsm::DevGraph g;
    g.n = n;
    g.nnz = nnz;
    g.row_ptr = d_row_ptr;
    g.col = d_col;
    g.labels = d_labels;
    g.rank = rank;
    g.piece_cnt = nullptr;
    g.tri_off = nullptr;
    g.tri_bits = nullptr;
    g.end_off = nullptr;
    e = fsm::launch_validate(g, num_labels, errw, st);
    int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, errw, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return err(FSM_ECUDA, std::string("validation: ") + cudaGetErrorString(e));
    if (bad) return err(FSM_EINVAL, "malformed CSR: rows must be sorted, symmetric, without self-loops or duplicates, labels in range");
    noalloc_rank_kernel<<<(unsigned)std::min<int64_t>(((int64_t)n + 255) / 256, 152 * 64), 256, 0, st>>>(d_labels, n, rank, cls);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = fsm::launch_level2_offsets(num_labels, cls, pair_off, total, st);
    if (e == cudaSuccess) e = fsm::launch_level2_domains(g, num_labels, pair_off, dom, pair_count, st);
    if (e == cudaSuccess)
        e = fsm::launch_level2_support(num_labels, cls, pair_off, dom, (unsigned long long *)d_support, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_count, pair_count, sizeof(uint64_t) * (size_t)num_labels * num_labels,
                            cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return err(FSM_ECUDA, std::string("edge supports: ") + cudaGetErrorString(e));
    return FSM_OK;
}
