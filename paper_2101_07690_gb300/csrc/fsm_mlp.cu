// fsm_mlp.cu -- the support-prediction network for sampled mining: 32 -> 64 -> 64 -> 1, ReLU,
// inputs standardised with stored means and deviations, BF16 weights in every forward and
// backward product, FP32 accumulation, FP32 master weights updated by Adam (Kingma and Ba,
// "Adam: a method for stochastic optimization", 2015), target log(MNI support).  All training
// and inference arithmetic runs in the kernels below; the host only orders minibatches.
//
// Parameter layout (FP32, 6337 values): W1[32][64] (input i, unit j), b1[64], W2[64][64],
// b2[64], w3[64], b3[1].
#include "fsm.h"
#include "fsm_kernels.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

namespace fsm {
void set_last_error_message(const std::string &m);
}

#define MLP_IN 32
#define MLP_H 64
#define MLP_NPARAM (MLP_IN * MLP_H + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1)
#define MLP_TILE 32   // samples per block

namespace {

constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + MLP_IN * MLP_H;
constexpr int OFF_W2 = OFF_B1 + MLP_H;
constexpr int OFF_B2 = OFF_W2 + MLP_H * MLP_H;
constexpr int OFF_W3 = OFF_B2 + MLP_H;
constexpr int OFF_B3 = OFF_W3 + MLP_H;

struct Smem {
    float w1[MLP_IN * MLP_H];
    float w2[MLP_H * MLP_H];
    float w3[MLP_H];
    float b1[MLP_H], b2[MLP_H];
    float x[MLP_TILE][MLP_IN];
    float h1[MLP_TILE][MLP_H];
    float h2[MLP_TILE][MLP_H];
    float dz[MLP_TILE][MLP_H];
    float y[MLP_TILE];
};

// stage BF16 weights (as float) and FP32 biases into shared memory; 64 threads
__device__ void stage_weights(Smem &s, const __nv_bfloat16 *wbf, const float *master) {
    for (int x = threadIdx.x; x < MLP_IN * MLP_H; x += blockDim.x) s.w1[x] = __bfloat162float(wbf[OFF_W1 + x]);
    for (int x = threadIdx.x; x < MLP_H * MLP_H; x += blockDim.x) s.w2[x] = __bfloat162float(wbf[OFF_W2 + x]);
    for (int x = threadIdx.x; x < MLP_H; x += blockDim.x) {
        s.w3[x] = __bfloat162float(wbf[OFF_W3 + x]);
        s.b1[x] = master[OFF_B1 + x];
        s.b2[x] = master[OFF_B2 + x];
    }
}

// forward over one tile (rows < nrows valid); thread j owns hidden unit j
__device__ void forward_tile(Smem &s, const float *X, const int64_t *rows, int64_t base, int nrows, const float *mu,
                             const float *sd, float b3) {
    const int j = threadIdx.x;
    for (int x = j; x < MLP_TILE * MLP_IN; x += blockDim.x) {
        const int r = x / MLP_IN, i = x % MLP_IN;
        float v = 0.f;
        if (r < nrows) {
            const int64_t row = rows ? rows[base + r] : base + r;
            v = (X[row * MLP_IN + i] - mu[i]) / sd[i];
        }
        s.x[r][i] = v;
    }
    __syncthreads();
    for (int r = 0; r < MLP_TILE; ++r) {
        float z = s.b1[j];
        for (int i = 0; i < MLP_IN; ++i) z = fmaf(s.x[r][i], s.w1[i * MLP_H + j], z);
        s.h1[r][j] = z;   // pre-activation kept; ReLU applied on use
    }
    __syncthreads();
    for (int r = 0; r < MLP_TILE; ++r) {
        float z = s.b2[j];
        for (int i = 0; i < MLP_H; ++i) z = fmaf(fmaxf(s.h1[r][i], 0.f), s.w2[i * MLP_H + j], z);
        s.h2[r][j] = z;
    }
    __syncthreads();
    if (j < MLP_TILE) {
        float z = b3;
        for (int i = 0; i < MLP_H; ++i) z = fmaf(fmaxf(s.h2[j][i], 0.f), s.w3[i], z);
        s.y[j] = z;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(MLP_H) infer_kernel(const float *X, int64_t n, const __nv_bfloat16 *wbf,
                                                      const float *master, const float *mu, const float *sd,
                                                      float *out) {
    extern __shared__ float smem_raw[];
    Smem &s = *reinterpret_cast<Smem *>(smem_raw);
    stage_weights(s, wbf, master);
    __syncthreads();
    const float b3 = master[OFF_B3];
    for (int64_t base = (int64_t)blockIdx.x * MLP_TILE; base < n; base += (int64_t)gridDim.x * MLP_TILE) {
        const int nrows = (int)(n - base < MLP_TILE ? n - base : MLP_TILE);
        forward_tile(s, X, nullptr, base, nrows, mu, sd, b3);
        if (threadIdx.x < nrows) out[base + threadIdx.x] = s.y[threadIdx.x];
        __syncthreads();
    }
}

// forward + backward of one minibatch (rows[base .. base+nb)); gradients of the mean squared
// error are added into grad (FP32); loss_sum gets the summed squared error
__global__ void __launch_bounds__(MLP_H) grad_kernel(const float *X, const float *Y, const int64_t *rows, int64_t base0,
                                                     int64_t nb, const __nv_bfloat16 *wbf, const float *master,
                                                     const float *mu, const float *sd, float *grad, float *loss_sum) {
    extern __shared__ float smem_raw[];
    Smem &s = *reinterpret_cast<Smem *>(smem_raw);
    stage_weights(s, wbf, master);
    __syncthreads();
    const float b3 = master[OFF_B3];
    const int j = threadIdx.x;
    const float inv = 1.f / (float)nb;
    for (int64_t t0 = (int64_t)blockIdx.x * MLP_TILE; t0 < nb; t0 += (int64_t)gridDim.x * MLP_TILE) {
        const int nrows = (int)(nb - t0 < MLP_TILE ? nb - t0 : MLP_TILE);
        forward_tile(s, X, rows, base0 + t0, nrows, mu, sd, b3);
        // dL/dy for the mean squared error, zero for padding rows
        if (j < MLP_TILE) {
            float d = 0.f;
            if (j < nrows) {
                const int64_t row = rows ? rows[base0 + t0 + j] : base0 + t0 + j;
                const float e = s.y[j] - Y[row];
                atomicAdd(loss_sum, e * e);
                d = 2.f * e * inv;
            }
            s.y[j] = d;
        }
        __syncthreads();
        // layer 3
        float gw3 = 0.f, gb3 = 0.f;
        for (int r = 0; r < MLP_TILE; ++r) {
            gw3 += s.y[r] * fmaxf(s.h2[r][j], 0.f);
            gb3 += s.y[r];
            s.dz[r][j] = s.h2[r][j] > 0.f ? s.y[r] * s.w3[j] : 0.f;   // dz2
        }
        atomicAdd(grad + OFF_W3 + j, gw3);
        if (j == 0) atomicAdd(grad + OFF_B3, gb3);
        __syncthreads();
        // layer 2: thread j is output unit j of W2
        float gb2 = 0.f;
        for (int r = 0; r < MLP_TILE; ++r) gb2 += s.dz[r][j];
        atomicAdd(grad + OFF_B2 + j, gb2);
        for (int i = 0; i < MLP_H; ++i) {
            float g = 0.f;
            for (int r = 0; r < MLP_TILE; ++r) g = fmaf(fmaxf(s.h1[r][i], 0.f), s.dz[r][j], g);
            atomicAdd(grad + OFF_W2 + i * MLP_H + j, g);
        }
        // dz1 (thread j now is hidden unit j of layer 1): dh1 = W2 dz2, masked by z1 > 0
        float dz1[MLP_TILE];
        for (int r = 0; r < MLP_TILE; ++r) {
            float d = 0.f;
            for (int o = 0; o < MLP_H; ++o) d = fmaf(s.w2[j * MLP_H + o], s.dz[r][o], d);
            dz1[r] = s.h1[r][j] > 0.f ? d : 0.f;
        }
        __syncthreads();
        for (int r = 0; r < MLP_TILE; ++r) s.dz[r][j] = dz1[r];
        __syncthreads();
        float gb1 = 0.f;
        for (int r = 0; r < MLP_TILE; ++r) gb1 += s.dz[r][j];
        atomicAdd(grad + OFF_B1 + j, gb1);
        for (int i = 0; i < MLP_IN; ++i) {
            float g = 0.f;
            for (int r = 0; r < MLP_TILE; ++r) g = fmaf(s.x[r][i], s.dz[r][j], g);
            atomicAdd(grad + OFF_W1 + i * MLP_H + j, g);
        }
        __syncthreads();
    }
}

__global__ void adam_kernel(float *w, float *m, float *v, const float *g, __nv_bfloat16 *wbf, int n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const float gx = g[x];
        const float mx = b1 * m[x] + (1.f - b1) * gx;
        const float vx = b2 * v[x] + (1.f - b2) * gx * gx;
        m[x] = mx;
        v[x] = vx;
        const float wx = w[x] - lr * (mx / c1) / (sqrtf(vx / c2) + eps);
        w[x] = wx;
        wbf[x] = __float2bfloat16_rn(wx);
    }
}

__global__ void to_bf16_kernel(const float *w, __nv_bfloat16 *wbf, int n) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
        wbf[x] = __float2bfloat16_rn(w[x]);
}

uint64_t host_mix(uint64_t &state) {
    uint64_t z = (state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// the kernels' shared memory exceeds the 48 KB default: opt in once per process and device
bool mlp_smem_ready() {
    static int done[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    if (done[dev]) return true;
    const int bytes = (int)sizeof(Smem);
    if (cudaFuncSetAttribute(infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) return false;
    if (cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) return false;
    done[dev] = 1;
    return true;
}

int mlp_fail(int code, const std::string &m) {
    fsm::set_last_error_message(m);
    return code;
}

} // namespace

struct fsm_mlp {
    float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr, *mu = nullptr, *sd = nullptr, *loss = nullptr;
    __nv_bfloat16 *wbf = nullptr;
    int64_t steps = 0;
};

namespace {
bool mlp_alloc(fsm_mlp *M) {
    const size_t P = MLP_NPARAM;
    return cudaMalloc(&M->w, P * 4) == cudaSuccess && cudaMalloc(&M->m, P * 4) == cudaSuccess &&
           cudaMalloc(&M->v, P * 4) == cudaSuccess && cudaMalloc(&M->g, P * 4) == cudaSuccess &&
           cudaMalloc(&M->mu, MLP_IN * 4) == cudaSuccess && cudaMalloc(&M->sd, MLP_IN * 4) == cudaSuccess &&
           cudaMalloc(&M->loss, 4) == cudaSuccess && cudaMalloc(&M->wbf, P * 2) == cudaSuccess;
}
} // namespace

extern "C" {

int fsm_mlp_create(uint64_t seed, fsm_mlp **out) {
    if (!out) return mlp_fail(FSM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!mlp_smem_ready()) return mlp_fail(FSM_ECUDA, "could not enable the network kernels' shared memory");
    fsm_mlp *M = new fsm_mlp();
    if (!mlp_alloc(M)) { fsm_mlp_free(M); return mlp_fail(FSM_ENOMEM, "device allocation for the network failed"); }
    // He-uniform initial weights from a splitmix64 stream, zero biases, identity standardisation
    std::vector<float> w(MLP_NPARAM, 0.f), mu(MLP_IN, 0.f), sd(MLP_IN, 1.f);
    uint64_t st = seed;
    auto uni = [&]() { return (float)((host_mix(st) >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f; };
    const float a1 = std::sqrt(6.f / MLP_IN), a2 = std::sqrt(6.f / MLP_H);
    for (int x = 0; x < MLP_IN * MLP_H; ++x) w[OFF_W1 + x] = a1 * uni();
    for (int x = 0; x < MLP_H * MLP_H; ++x) w[OFF_W2 + x] = a2 * uni();
    for (int x = 0; x < MLP_H; ++x) w[OFF_W3 + x] = a2 * uni();
    int rc = fsm_mlp_set_params(M, w.data());
    if (rc == FSM_OK) rc = fsm_mlp_set_norm(M, mu.data(), sd.data());
    if (rc != FSM_OK) { fsm_mlp_free(M); return rc; }
    *out = M;
    return FSM_OK;
}

int fsm_mlp_set_params(fsm_mlp *M, const float *params) {
    if (!M || !params) return mlp_fail(FSM_EINVAL, "NULL argument");
    const size_t P = MLP_NPARAM;
    cudaError_t e = cudaMemcpy(M->w, params, P * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(M->m, 0, P * 4);
    if (e == cudaSuccess) e = cudaMemset(M->v, 0, P * 4);
    if (e == cudaSuccess) {
        to_bf16_kernel<<<(MLP_NPARAM + 255) / 256, 256>>>(M->w, M->wbf, MLP_NPARAM);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    M->steps = 0;
    return e == cudaSuccess ? FSM_OK : mlp_fail(FSM_ECUDA, cudaGetErrorString(e));
}

int fsm_mlp_get_params(const fsm_mlp *M, float *params) {
    if (!M || !params) return mlp_fail(FSM_EINVAL, "NULL argument");
    cudaError_t e = cudaMemcpy(params, M->w, (size_t)MLP_NPARAM * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? FSM_OK : mlp_fail(FSM_ECUDA, cudaGetErrorString(e));
}

int fsm_mlp_set_norm(fsm_mlp *M, const float *mean, const float *stdev) {
    if (!M || !mean || !stdev) return mlp_fail(FSM_EINVAL, "NULL argument");
    for (int i = 0; i < MLP_IN; ++i)
        if (!(stdev[i] > 0.f)) return mlp_fail(FSM_EINVAL, "standard deviations must be positive");
    cudaError_t e = cudaMemcpy(M->mu, mean, MLP_IN * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(M->sd, stdev, MLP_IN * 4, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? FSM_OK : mlp_fail(FSM_ECUDA, cudaGetErrorString(e));
}

// Input standardisation from data: one block per input column, mean then the mean squared
// deviation (population), both accumulated in double; stdev floored at 1e-3.
__global__ void fit_norm_kernel(const float *X, int64_t n, float *mu, float *sd) {
    __shared__ double part[256];
    const int c = blockIdx.x;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)X[i * MLP_IN + c];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    const double mean = part[0] / (double)n;
    __syncthreads();
    double q = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double d = (double)X[i * MLP_IN + c] - mean;
        q += d * d;
    }
    part[threadIdx.x] = q;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        mu[c] = (float)mean;
        sd[c] = (float)fmax(sqrt(part[0] / (double)n), 1e-3);
    }
}

static int mlp_upload(const float *X, const float *Y, int64_t n, float **dX, float **dY);

int fsm_mlp_fit_norm(fsm_mlp *M, const float *X, int64_t n) {
    if (!M || !X || n < 1) return mlp_fail(FSM_EINVAL, "NULL argument or n < 1");
    float *dX = nullptr;
    int rc = mlp_upload(X, nullptr, n, &dX, nullptr);
    if (rc == FSM_OK) {
        fit_norm_kernel<<<MLP_IN, 256>>>(dX, n, M->mu, M->sd);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = mlp_fail(FSM_ECUDA, cudaGetErrorString(e));
    } else {
        rc = mlp_fail(rc, "could not stage the inputs on the device");
    }
    cudaFree(dX);
    return rc;
}

static int mlp_upload(const float *X, const float *Y, int64_t n, float **dX, float **dY) {
    *dX = nullptr;
    if (dY) *dY = nullptr;
    if (cudaMalloc(dX, (size_t)std::max<int64_t>(n, 1) * MLP_IN * 4) != cudaSuccess) return FSM_ENOMEM;
    if (dY && cudaMalloc(dY, (size_t)std::max<int64_t>(n, 1) * 4) != cudaSuccess) return FSM_ENOMEM;
    if (n && cudaMemcpy(*dX, X, (size_t)n * MLP_IN * 4, cudaMemcpyHostToDevice) != cudaSuccess) return FSM_ECUDA;
    if (dY && n && cudaMemcpy(*dY, Y, (size_t)n * 4, cudaMemcpyHostToDevice) != cudaSuccess) return FSM_ECUDA;
    return FSM_OK;
}

int fsm_mlp_gradients(fsm_mlp *M, const float *X, const float *Y, int64_t n, float *grads, float *loss) {
    if (!mlp_smem_ready()) return mlp_fail(FSM_ECUDA, "could not enable the network kernels' shared memory");
    if (!M || !X || !Y || !grads || n < 1) return mlp_fail(FSM_EINVAL, "NULL argument or n < 1");
    float *dX = nullptr, *dY = nullptr;
    int rc = mlp_upload(X, Y, n, &dX, &dY);
    if (rc == FSM_OK) {
        cudaMemset(M->g, 0, (size_t)MLP_NPARAM * 4);
        cudaMemset(M->loss, 0, 4);
        const int grid = (int)std::min<int64_t>((n + MLP_TILE - 1) / MLP_TILE, 4096);
        grad_kernel<<<grid, MLP_H, sizeof(Smem)>>>(dX, dY, nullptr, 0, n, M->wbf, M->w, M->mu, M->sd, M->g, M->loss);
        fsm::note_launches(1);
        float ls = 0.f;
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpy(grads, M->g, (size_t)MLP_NPARAM * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(&ls, M->loss, 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = mlp_fail(FSM_ECUDA, cudaGetErrorString(e));
        else if (loss) *loss = ls / (float)n;
    } else {
        rc = mlp_fail(rc, "could not stage the training data on the device");
    }
    cudaFree(dX);
    cudaFree(dY);
    return rc;
}

int fsm_mlp_train(fsm_mlp *M, const float *X, const float *Y, int64_t n, int32_t epochs, int32_t batch, float lr,
                  uint64_t seed, float *final_loss) {
    if (!mlp_smem_ready()) return mlp_fail(FSM_ECUDA, "could not enable the network kernels' shared memory");
    if (!M || !X || !Y || n < 1 || epochs < 1 || batch < 1 || !(lr > 0.f))
        return mlp_fail(FSM_EINVAL, "bad training arguments");
    float *dX = nullptr, *dY = nullptr;
    int64_t *drows = nullptr;
    int rc = mlp_upload(X, Y, n, &dX, &dY);
    if (rc == FSM_OK && cudaMalloc(&drows, (size_t)n * 8) != cudaSuccess) rc = FSM_ENOMEM;
    if (rc != FSM_OK) {
        cudaFree(dX); cudaFree(dY); cudaFree(drows);
        return mlp_fail(rc, "could not stage the training data on the device");
    }
    std::vector<int64_t> order((size_t)n);
    for (int64_t i = 0; i < n; ++i) order[(size_t)i] = i;
    uint64_t st = seed;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float epoch_loss = 0.f;
    cudaError_t e = cudaSuccess;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        for (int64_t i = n - 1; i > 0; --i) std::swap(order[(size_t)i], order[(size_t)(host_mix(st) % (uint64_t)(i + 1))]);
        e = cudaMemcpy(drows, order.data(), (size_t)n * 8, cudaMemcpyHostToDevice);
        cudaMemset(M->loss, 0, 4);
        for (int64_t b0 = 0; b0 < n && e == cudaSuccess; b0 += batch) {
            const int64_t nb = std::min<int64_t>(batch, n - b0);
            cudaMemset(M->g, 0, (size_t)MLP_NPARAM * 4);
            const int grid = (int)std::min<int64_t>((nb + MLP_TILE - 1) / MLP_TILE, 1024);
            grad_kernel<<<grid, MLP_H, sizeof(Smem)>>>(dX, dY, drows, b0, nb, M->wbf, M->w, M->mu, M->sd, M->g, M->loss);
            M->steps += 1;
            const float c1 = 1.f - std::pow(b1, (float)M->steps), c2 = 1.f - std::pow(b2, (float)M->steps);
            adam_kernel<<<(MLP_NPARAM + 255) / 256, 256>>>(M->w, M->m, M->v, M->g, M->wbf, MLP_NPARAM, lr, b1, b2, eps, c1, c2);
            fsm::note_launches(2);
            e = cudaGetLastError();
        }
        float ls = 0.f;
        if (e == cudaSuccess) e = cudaMemcpy(&ls, M->loss, 4, cudaMemcpyDeviceToHost);
        epoch_loss = ls / (float)n;
    }
    cudaFree(dX); cudaFree(dY); cudaFree(drows);
    if (e != cudaSuccess) return mlp_fail(FSM_ECUDA, cudaGetErrorString(e));
    if (final_loss) *final_loss = epoch_loss;
    return FSM_OK;
}

int fsm_mlp_predict(const fsm_mlp *M, const float *X, int64_t n, float *out) {
    if (!M || !X || !out || n < 0) return mlp_fail(FSM_EINVAL, "NULL argument");
    if (n == 0) return FSM_OK;
    float *dX = nullptr, *dO = nullptr;
    int rc = mlp_upload(X, nullptr, n, &dX, nullptr);
    if (rc == FSM_OK && cudaMalloc(&dO, (size_t)n * 4) != cudaSuccess) rc = FSM_ENOMEM;
    if (rc == FSM_OK) rc = fsm_mlp_predict_device(M, dX, n, dO, nullptr);
    if (rc == FSM_OK && cudaMemcpy(out, dO, (size_t)n * 4, cudaMemcpyDeviceToHost) != cudaSuccess) rc = FSM_ECUDA;
    cudaFree(dX);
    cudaFree(dO);
    return rc == FSM_OK ? FSM_OK : mlp_fail(rc, "prediction failed");
}

int fsm_mlp_predict_device(const fsm_mlp *M, const float *d_X, int64_t n, float *d_out, void *stream) {
    if (!mlp_smem_ready()) return mlp_fail(FSM_ECUDA, "could not enable the network kernels' shared memory");
    if (!M || !d_X || !d_out || n < 0) return mlp_fail(FSM_EINVAL, "NULL argument");
    if (n == 0) return FSM_OK;
    const int grid = (int)std::min<int64_t>((n + MLP_TILE - 1) / MLP_TILE, 2048);
    infer_kernel<<<grid, MLP_H, sizeof(Smem), (cudaStream_t)stream>>>(d_X, n, M->wbf, M->w, M->mu, M->sd, d_out);
    fsm::note_launches(1);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FSM_OK : mlp_fail(FSM_ECUDA, cudaGetErrorString(e));
}

void fsm_mlp_free(fsm_mlp *M) {
    if (!M) return;
    cudaFree(M->w); cudaFree(M->m); cudaFree(M->v); cudaFree(M->g);
    cudaFree(M->mu); cudaFree(M->sd); cudaFree(M->loss); cudaFree(M->wbf);
    delete M;
}

} // extern "C"
