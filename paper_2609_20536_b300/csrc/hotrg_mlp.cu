// Surrogate network kernels: an ensemble of 2 -> 128 -> 128 -> 128 -> 4 MLPs
// (tanh hidden layers, linear output) mapping (beta, Delta) to standardised
// (f, C_V, chi, chi1).  Weights are held in BF16 for the forward and
// backward products (FP32 master copies for Adam); every product accumulates
// in FP32.  Ensemble members run side by side (grid y = member).
//
//   forward:   h_l = tanh(h_{l-1} W_l + b_l), y = h_3 W_4 + b_4   (W stored [in][out])
//   loss:      mean squared error over the batch and the 4 outputs
//   backward:  g_y = 2 (y - t)/(n k); gW = h^T g; gb = sum_rows g; g_h = g W^T (1 - h^2)
//   Adam:      m, v moments, bias correction, FP32 master, BF16 copy refreshed
// Reductions over the batch are done in a fixed order (no atomics), so
// training is deterministic.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace hotrg {

constexpr int MLP_L = 4;
constexpr int MLP_SIZES[MLP_L + 1] = {2, 128, 128, 128, 4};
constexpr int MLP_MAXB = 4096;  // largest minibatch / prediction chunk

__host__ __device__ constexpr int mlp_in(int l) { return l == 0 ? 2 : 128; }
__host__ __device__ constexpr int mlp_out(int l) { return l == MLP_L - 1 ? 4 : 128; }
__host__ __device__ constexpr int64_t mlp_wcount(int l) { return (int64_t)mlp_in(l) * mlp_out(l); }

static int64_t mlp_layer_offset(int l) {  // offset of W_l in the flat [W_0 b_0 W_1 b_1 ...] layout
    int64_t o = 0;
    for (int i = 0; i < l; ++i) o += mlp_wcount(i) + mlp_out(i);
    return o;
}
static int64_t mlp_nparams() { return mlp_layer_offset(MLP_L); }

constexpr int MLP_ROWS = 16;  // batch rows per block

// out[n][o] = act(sum_i in[n][i] W[i][o] + b[o]) for MLP_ROWS rows of member e
__global__ void __launch_bounds__(128) mlp_fwd_kernel(const float* __restrict__ in, int64_t in_mstride, int in_dim,
                                                      const __nv_bfloat16* __restrict__ W, int64_t w_mstride,
                                                      const float* __restrict__ b, int64_t b_mstride, int out_dim,
                                                      float* __restrict__ out, int64_t out_mstride, int n, int act) {
    __shared__ __nv_bfloat16 Ws[128 * 128];
    __shared__ float xs[MLP_ROWS][129];
    const int e = blockIdx.y;
    in += e * in_mstride;
    W += e * w_mstride;
    b += e * b_mstride;
    out += e * out_mstride;
    const int n0 = blockIdx.x * MLP_ROWS;
    for (int i = threadIdx.x; i < in_dim * out_dim; i += blockDim.x) Ws[i] = W[i];
    for (int i = threadIdx.x; i < MLP_ROWS * in_dim; i += blockDim.x) {
        const int r = i / in_dim, c = i % in_dim;
        xs[r][c] = (n0 + r < n) ? in[(int64_t)(n0 + r) * in_dim + c] : 0.f;
    }
    __syncthreads();
    const int o = threadIdx.x;
    if (o < out_dim) {
        for (int r = 0; r < MLP_ROWS && n0 + r < n; ++r) {
            float acc = b[o];
            for (int i = 0; i < in_dim; ++i) acc = fmaf(xs[r][i], __bfloat162float(Ws[i * out_dim + o]), acc);
            out[(int64_t)(n0 + r) * out_dim + o] = act ? tanhf(acc) : acc;
        }
    }
}

// g = 2 (y - t) / (n k), per-member loss partials
__global__ void mlp_loss_grad_kernel(const float* __restrict__ y, int64_t y_mstride, const float* __restrict__ t,
                                     int n, float* __restrict__ g, float* __restrict__ loss_part) {
    __shared__ float sh[256];
    const int e = blockIdx.y;
    y += e * y_mstride;
    g += e * y_mstride;
    const int k = 4;
    float s = 0.f;
    for (int i = threadIdx.x; i < n * k; i += blockDim.x) {
        const float d = y[i] - t[i];
        g[i] = 2.f * d / (float)(n * k);
        s += d * d;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[e] = sh[0] / (float)(n * k);
}

// gW[i][o] = sum_n h[n][i] g[n][o], gb[o] = sum_n g[n][o]  (block per 32 inputs i, threads over o)
__global__ void __launch_bounds__(128) mlp_wgrad_kernel(const float* __restrict__ h, int64_t h_mstride, int in_dim,
                                                        const float* __restrict__ g, int64_t g_mstride, int out_dim,
                                                        int n, float* __restrict__ gW, float* __restrict__ gb,
                                                        int64_t p_mstride) {
    __shared__ float hs[32][33];
    __shared__ float gs[32][129];
    const int e = blockIdx.y;
    h += e * h_mstride;
    g += e * g_mstride;
    gW += e * p_mstride;
    gb += e * p_mstride;
    const int i0 = blockIdx.x * 32;
    const int o = threadIdx.x;
    float acc[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) acc[r] = 0.f;
    float bacc = 0.f;
    for (int n0 = 0; n0 < n; n0 += 32) {
        for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
            const int rn = idx / 32, ci = idx % 32;
            hs[rn][ci] = (n0 + rn < n && i0 + ci < in_dim) ? h[(int64_t)(n0 + rn) * in_dim + i0 + ci] : 0.f;
        }
        for (int idx = threadIdx.x; idx < 32 * out_dim; idx += blockDim.x) {
            const int rn = idx / out_dim, co = idx % out_dim;
            gs[rn][co] = (n0 + rn < n) ? g[(int64_t)(n0 + rn) * out_dim + co] : 0.f;
        }
        __syncthreads();
        if (o < out_dim) {
            for (int rn = 0; rn < 32; ++rn) {
                const float gv = gs[rn][o];
                bacc += gv;
#pragma unroll
                for (int ci = 0; ci < 32; ++ci) acc[ci] = fmaf(hs[rn][ci], gv, acc[ci]);
            }
        }
        __syncthreads();
    }
    if (o < out_dim) {
#pragma unroll
        for (int ci = 0; ci < 32; ++ci)
            if (i0 + ci < in_dim) gW[(int64_t)(i0 + ci) * out_dim + o] = acc[ci];
        if (blockIdx.x == 0) gb[o] = bacc;
    }
}

// gin[n][i] = (sum_o g[n][o] W[i][o]) (1 - h[n][i]^2)   (h = this layer's input, a tanh output)
__global__ void __launch_bounds__(128) mlp_ingrad_kernel(const float* __restrict__ g, int64_t g_mstride, int out_dim,
                                                         const __nv_bfloat16* __restrict__ W, int64_t w_mstride,
                                                         int in_dim, const float* __restrict__ h, int64_t h_mstride,
                                                         float* __restrict__ gin, int n) {
    __shared__ __nv_bfloat16 Ws[128 * 128];
    __shared__ float gsh[MLP_ROWS][129];
    const int e = blockIdx.y;
    g += e * g_mstride;
    W += e * w_mstride;
    h += e * h_mstride;
    gin += e * h_mstride;
    const int n0 = blockIdx.x * MLP_ROWS;
    for (int i = threadIdx.x; i < in_dim * out_dim; i += blockDim.x) Ws[i] = W[i];
    for (int i = threadIdx.x; i < MLP_ROWS * out_dim; i += blockDim.x) {
        const int r = i / out_dim, c = i % out_dim;
        gsh[r][c] = (n0 + r < n) ? g[(int64_t)(n0 + r) * out_dim + c] : 0.f;
    }
    __syncthreads();
    const int i = threadIdx.x;
    if (i < in_dim) {
        for (int r = 0; r < MLP_ROWS && n0 + r < n; ++r) {
            float acc = 0.f;
            for (int o = 0; o < out_dim; ++o) acc = fmaf(gsh[r][o], __bfloat162float(Ws[i * out_dim + o]), acc);
            const float hv = h[(int64_t)(n0 + r) * in_dim + i];
            gin[(int64_t)(n0 + r) * in_dim + i] = acc * (1.f - hv * hv);
        }
    }
}

__global__ void mlp_adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, __nv_bfloat16* __restrict__ wb, int64_t np, float lr,
                                float b1, float b2, float eps, float c1, float c2, const int32_t* __restrict__ is_w) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        wb[i] = __float2bfloat16_rn(wi);
    }
    (void)is_w;
}

__global__ void mlp_to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, int64_t np) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x)
        wb[i] = __float2bfloat16_rn(w[i]);
}

// mean and spread (standard deviation) over the ensemble: y is [E][n][4]
__global__ void mlp_ensemble_stats_kernel(const float* __restrict__ y, int E, int64_t n4, float* __restrict__ mean,
                                          float* __restrict__ spread) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f, s2 = 0.f;
        for (int e = 0; e < E; ++e) {
            const float v = y[(int64_t)e * n4 + i];
            s += v;
            s2 += v * v;
        }
        const float mu = s / E;
        mean[i] = mu;
        spread[i] = E > 1 ? sqrtf(fmaxf(s2 / E - mu * mu, 0.f)) : 0.f;
    }
}

}  // namespace hotrg

using namespace hotrg;

struct hotrg_mlp {
    cudaStream_t stream = nullptr;
    int E = 1;
    int64_t np = 0;
    float* w = nullptr;          // [E][np] FP32 master
    __nv_bfloat16* wb = nullptr; // [E][np] BF16 copy used by the products
    float* g = nullptr;          // [E][np] gradients
    float* m = nullptr;
    float* v = nullptr;
    float* act = nullptr;        // activations [E][L+1][MAXB][128]
    float* gbuf = nullptr;       // [E][2][MAXB][128] backward scratch
    float* x = nullptr;          // [MAXB][2]
    float* t = nullptr;          // [MAXB][4]
    float* loss = nullptr;       // [E]
    float* ymean = nullptr;      // [MAXB][4]
    float* yspread = nullptr;
    int64_t steps = 0;
    uint64_t seed = 0;
};

namespace {

constexpr int64_t ACT_STRIDE = (int64_t)MLP_MAXB * 128;  // one layer's activations

float* act_ptr(hotrg_mlp* m, int l) { return m->act + (int64_t)l * ACT_STRIDE; }
int64_t act_mstride() { return (int64_t)(MLP_L + 1) * ACT_STRIDE; }

void forward(hotrg_mlp* m, const float* x_dev, int n) {
    // layer 0 input is x (shared by all members): copy into every member's h_0
    for (int e = 0; e < m->E; ++e)
        cudaMemcpyAsync(m->act + e * act_mstride(), x_dev, sizeof(float) * n * 2, cudaMemcpyDeviceToDevice,
                        m->stream);
    for (int l = 0; l < MLP_L; ++l) {
        const int64_t wo = mlp_layer_offset(l);
        dim3 grid((n + MLP_ROWS - 1) / MLP_ROWS, m->E);
        mlp_fwd_kernel<<<grid, 128, 0, m->stream>>>(act_ptr(m, l), act_mstride(), mlp_in(l), m->wb + wo, m->np,
                                                   m->w + wo + mlp_wcount(l), m->np, mlp_out(l),
                                                   act_ptr(m, l + 1), act_mstride(), n, l < MLP_L - 1 ? 1 : 0);
        HOTRG_COUNT(1);
    }
}

void backward(hotrg_mlp* m, const float* t_dev, int n) {
    float* y = act_ptr(m, MLP_L);
    float* g0 = m->gbuf;
    const int64_t gstride = 2 * ACT_STRIDE;
    float* g1 = m->gbuf + ACT_STRIDE;
    dim3 one(1, m->E);
    mlp_loss_grad_kernel<<<one, 256, 0, m->stream>>>(y, act_mstride(), t_dev, n, g0, m->loss);
    // note: mlp_loss_grad writes g with member stride act_mstride(); keep gradients in the activation-strided
    // layout by aliasing g0 = gbuf with the same stride
    HOTRG_COUNT(1);
    float* gcur = g0;
    float* gnext = g1;
    for (int l = MLP_L - 1; l >= 0; --l) {
        const int64_t wo = mlp_layer_offset(l);
        dim3 gw((mlp_in(l) + 31) / 32, m->E);
        mlp_wgrad_kernel<<<gw, 128, 0, m->stream>>>(act_ptr(m, l), act_mstride(), mlp_in(l), gcur, act_mstride(),
                                                   mlp_out(l), n, m->g + wo, m->g + wo + mlp_wcount(l), m->np);
        HOTRG_COUNT(1);
        if (l > 0) {
            dim3 gi((n + MLP_ROWS - 1) / MLP_ROWS, m->E);
            mlp_ingrad_kernel<<<gi, 128, 0, m->stream>>>(gcur, act_mstride(), mlp_out(l), m->wb + wo, m->np,
                                                         mlp_in(l), act_ptr(m, l), act_mstride(), gnext, n);
            HOTRG_COUNT(1);
            float* tmp = gcur;
            gcur = gnext;
            gnext = tmp;
        }
    }
    (void)gstride;
}

void adam(hotrg_mlp* m, float lr) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    m->steps += 1;
    const float c1 = 1.f - powf(b1, (float)m->steps), c2 = 1.f - powf(b2, (float)m->steps);
    const int64_t tot = m->np * m->E;
    mlp_adam_kernel<<<296, 256, 0, m->stream>>>(m->w, m->g, m->m, m->v, m->wb, tot, lr, b1, b2, eps, c1, c2,
                                                nullptr);
    HOTRG_COUNT(1);
}

// deterministic Glorot-uniform initialisation on the host (splitmix64 stream per member)
uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" {

hotrg_status hotrg_mlp_create(hotrg_mlp** out, int32_t ensemble, uint64_t seed, void* cuda_stream) {
    if (!out || ensemble < 1 || ensemble > 16) return HOTRG_EINVAL;
    *out = nullptr;
    hotrg_mlp* m = new hotrg_mlp();
    m->stream = (cudaStream_t)cuda_stream;
    m->E = ensemble;
    m->np = mlp_nparams();
    m->seed = seed;
    const int64_t P = m->np * m->E;
    bool ok = cudaMalloc(&m->w, P * 4) == cudaSuccess && cudaMalloc(&m->wb, P * 2) == cudaSuccess &&
              cudaMalloc(&m->g, P * 4) == cudaSuccess && cudaMalloc(&m->m, P * 4) == cudaSuccess &&
              cudaMalloc(&m->v, P * 4) == cudaSuccess &&
              cudaMalloc(&m->act, act_mstride() * m->E * 4) == cudaSuccess &&
              cudaMalloc(&m->gbuf, act_mstride() * m->E * 4) == cudaSuccess &&
              cudaMalloc(&m->x, (int64_t)MLP_MAXB * 2 * 4) == cudaSuccess &&
              cudaMalloc(&m->t, (int64_t)MLP_MAXB * 4 * 4) == cudaSuccess &&
              cudaMalloc(&m->loss, 64 * 4) == cudaSuccess &&
              cudaMalloc(&m->ymean, (int64_t)MLP_MAXB * 4 * 4) == cudaSuccess &&
              cudaMalloc(&m->yspread, (int64_t)MLP_MAXB * 4 * 4) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        hotrg_mlp_destroy(m);
        return HOTRG_ENOMEM;
    }
    // Glorot-uniform weights, zero biases, per member from its own stream of the seed
    std::vector<float> h(P);
    for (int e = 0; e < m->E; ++e) {
        uint64_t s = seed * 0x100000001B3ull + (uint64_t)e * 0x9E3779B97F4A7C15ull + 1;
        for (int l = 0; l < MLP_L; ++l) {
            const int64_t wo = mlp_layer_offset(l);
            const float lim = sqrtf(6.f / (float)(mlp_in(l) + mlp_out(l)));
            for (int64_t i = 0; i < mlp_wcount(l); ++i)
                h[e * m->np + wo + i] = lim * (2.f * (float)((splitmix(s) >> 11) * (1.0 / 9007199254740992.0)) - 1.f);
            for (int i = 0; i < mlp_out(l); ++i) h[e * m->np + wo + mlp_wcount(l) + i] = 0.f;
        }
    }
    cudaMemcpy(m->w, h.data(), P * 4, cudaMemcpyHostToDevice);
    cudaMemset(m->m, 0, P * 4);
    cudaMemset(m->v, 0, P * 4);
    mlp_to_bf16_kernel<<<296, 256, 0, m->stream>>>(m->w, m->wb, P);
    HOTRG_COUNT(1);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
        cudaGetLastError();
        hotrg_mlp_destroy(m);
        return HOTRG_ECUDA;
    }
    *out = m;
    return HOTRG_OK;
}

void hotrg_mlp_destroy(hotrg_mlp* m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    void* ptrs[] = {m->w, m->wb, m->g, m->m, m->v, m->act, m->gbuf, m->x, m->t, m->loss, m->ymean, m->yspread};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete m;
}

int64_t hotrg_mlp_num_params(void) { return mlp_nparams(); }

hotrg_status hotrg_mlp_set_params(hotrg_mlp* m, int32_t member, const float* flat) {
    if (!m || !flat || member < 0 || member >= m->E) return HOTRG_EINVAL;
    if (cudaMemcpyAsync(m->w + member * m->np, flat, m->np * 4, cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
        return HOTRG_ECUDA;
    mlp_to_bf16_kernel<<<296, 256, 0, m->stream>>>(m->w + member * m->np, m->wb + member * m->np, m->np);
    HOTRG_COUNT(1);
    return cudaStreamSynchronize(m->stream) == cudaSuccess ? HOTRG_OK : HOTRG_ECUDA;
}

hotrg_status hotrg_mlp_get_params(hotrg_mlp* m, int32_t member, float* flat) {
    if (!m || !flat || member < 0 || member >= m->E) return HOTRG_EINVAL;
    if (cudaMemcpyAsync(flat, m->w + member * m->np, m->np * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
        return HOTRG_ECUDA;
    return cudaStreamSynchronize(m->stream) == cudaSuccess ? HOTRG_OK : HOTRG_ECUDA;
}

hotrg_status hotrg_mlp_gradients(hotrg_mlp* m, int32_t member, const float* X, const float* T, int32_t n,
                                 float* loss, float* grad_flat) {
    if (!m || !X || !T || n < 1 || n > MLP_MAXB || member < 0 || member >= m->E) return HOTRG_EINVAL;
    cudaMemcpyAsync(m->x, X, (int64_t)n * 2 * 4, cudaMemcpyHostToDevice, m->stream);
    cudaMemcpyAsync(m->t, T, (int64_t)n * 4 * 4, cudaMemcpyHostToDevice, m->stream);
    forward(m, m->x, n);
    backward(m, m->t, n);
    if (grad_flat)
        cudaMemcpyAsync(grad_flat, m->g + member * m->np, m->np * 4, cudaMemcpyDeviceToHost, m->stream);
    float lh[64];
    cudaMemcpyAsync(lh, m->loss, m->E * 4, cudaMemcpyDeviceToHost, m->stream);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
        cudaGetLastError();
        return HOTRG_ECUDA;
    }
    if (loss) *loss = lh[member];
    return HOTRG_OK;
}

hotrg_status hotrg_mlp_train(hotrg_mlp* m, const float* X, const float* T, int32_t n, int32_t epochs, int32_t batch,
                             float lr, float* final_loss) {
    if (!m || !X || !T || n < 1 || epochs < 0 || batch < 1 || batch > MLP_MAXB || !(lr > 0.f)) return HOTRG_EINVAL;
    // minibatches drawn from a per-epoch permutation (host, deterministic)
    std::vector<float> bx((size_t)batch * 2), bt((size_t)batch * 4);
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    std::vector<float> hX(X, X + (size_t)n * 2), hT(T, T + (size_t)n * 4);
    uint64_t s = m->seed ^ 0xD1B54A32D192ED03ull;
    float last = 0.f;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int i = n - 1; i > 0; --i) {
            const int j = (int)(splitmix(s) % (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        for (int b0 = 0; b0 < n; b0 += batch) {
            const int nb = std::min(batch, n - b0);
            for (int r = 0; r < nb; ++r) {
                memcpy(&bx[(size_t)r * 2], &hX[(size_t)perm[b0 + r] * 2], 8);
                memcpy(&bt[(size_t)r * 4], &hT[(size_t)perm[b0 + r] * 4], 16);
            }
            cudaMemcpyAsync(m->x, bx.data(), (int64_t)nb * 2 * 4, cudaMemcpyHostToDevice, m->stream);
            cudaMemcpyAsync(m->t, bt.data(), (int64_t)nb * 4 * 4, cudaMemcpyHostToDevice, m->stream);
            forward(m, m->x, nb);
            backward(m, m->t, nb);
            adam(m, lr);
            cudaStreamSynchronize(m->stream);  // the host staging buffers are reused
        }
    }
    float lh[64];
    cudaMemcpyAsync(lh, m->loss, m->E * 4, cudaMemcpyDeviceToHost, m->stream);
    const cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return HOTRG_ECUDA;
    }
    for (int i = 0; i < m->E; ++i) last += lh[i] / m->E;
    if (final_loss) *final_loss = last;
    return HOTRG_OK;
}

hotrg_status hotrg_mlp_predict(hotrg_mlp* m, const float* X, int32_t n, float* mean, float* spread) {
    if (!m || !X || !mean || n < 0) return HOTRG_EINVAL;
    for (int b0 = 0; b0 < n; b0 += MLP_MAXB) {
        const int nb = std::min(MLP_MAXB, n - b0);
        cudaMemcpyAsync(m->x, X + (size_t)b0 * 2, (int64_t)nb * 2 * 4, cudaMemcpyHostToDevice, m->stream);
        forward(m, m->x, nb);
        // gather the members' outputs [E][nb][4] into a contiguous buffer (reuse gbuf)
        for (int e = 0; e < m->E; ++e)
            cudaMemcpyAsync(m->gbuf + (int64_t)e * nb * 4, act_ptr(m, MLP_L) + e * act_mstride(),
                            (int64_t)nb * 4 * 4, cudaMemcpyDeviceToDevice, m->stream);
        mlp_ensemble_stats_kernel<<<64, 256, 0, m->stream>>>(m->gbuf, m->E, (int64_t)nb * 4, m->ymean, m->yspread);
        HOTRG_COUNT(1);
        cudaMemcpyAsync(mean + (size_t)b0 * 4, m->ymean, (int64_t)nb * 4 * 4, cudaMemcpyDeviceToHost, m->stream);
        if (spread)
            cudaMemcpyAsync(spread + (size_t)b0 * 4, m->yspread, (int64_t)nb * 4 * 4, cudaMemcpyDeviceToHost,
                            m->stream);
        if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
            cudaGetLastError();
            return HOTRG_ECUDA;
        }
    }
    return HOTRG_OK;
}

}  // extern "C"
