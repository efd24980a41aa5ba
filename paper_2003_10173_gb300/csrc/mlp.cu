// Learned rank model: a 3-layer perceptron (8 -> 64 -> 64 -> 1, GELU) that predicts, per
// tree level, the probe count the adaptive range finder settles on (Section 3.3: the
// per-level sample count is the quantity being tuned), so that peeling can start there.
//
// Kernels:
//   rm_train_kernel    one CTA runs `steps` Adam steps back to back: per minibatch, chunks of
//                      64 rows go through the forward pass, the backward pass (gradients
//                      accumulated in registers, fixed summation order) and, after the last
//                      chunk, the Adam update of the FP32 master weights held in shared
//                      memory.  The whole training state (master weights, both moments, the
//                      effective weights and one chunk's activations, ~182 KB) stays in shared
//                      memory for the launch.  With grad_only the kernel returns the loss and
//                      gradient of one full pass instead of updating.
//   rm_predict_kernel  one CTA per 64 rows, forward pass only.
//   rm_init_kernel     U(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights from the counter-based
//                      generator, zero biases.
// Arithmetic is FP32; with bf16 the forward and backward passes use the master weights
// rounded to bfloat16 (nearest even), refreshed after every update.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>

#include "handle.h"

struct h2_rankmodel_s {
    int device = 0;
    int bf16 = 1;
    uint64_t seed = 0;
    int64_t step = 0;
    h2::DevBuf<float> params, adam_m, adam_v;
    h2::DevBuf<float> grad, loss, feat, pred;
    h2::DevBuf<int> err;   // set by the training kernel on a minibatch index outside [0, n)
};

namespace h2 {

namespace {

constexpr int F = H2_RM_FEATURES;
constexpr int HW = H2_RM_WIDTH;
constexpr int NP = H2_RM_NPARAM;
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + HW * F;
constexpr int OFF_W2 = OFF_B1 + HW;
constexpr int OFF_B2 = OFF_W2 + HW * HW;
constexpr int OFF_W3 = OFF_B2 + HW;
constexpr int OFF_B3 = OFF_W3 + HW;
static_assert(OFF_B3 + 1 == NP, "parameter layout");
static_assert(F == 8 && HW == 64, "the thread mappings below assume 8 features and width 64");

constexpr int NT = 256;        // threads of every MLP kernel
constexpr int CS = 64;         // rows per chunk
constexpr int LDA = HW + 1;    // padded row stride of the activation tiles
constexpr int STREAM_MLP_INIT = 6;
constexpr int STREAM_MLP_DATA = 7;
constexpr int MAX_BATCH = 1024;

constexpr float BETA1 = 0.9f, BETA2 = 0.999f, ADAM_EPS = 1e-8f;
constexpr float C_GELU = 0.7978845608028654f;   // sqrt(2/pi)

// shared-memory layout (floats)
constexpr int SM_W = 0;                       // effective weights, parameter layout
constexpr int SM_W2T = SM_W + NP + 3;         // effective W2 transposed: [i][o]
constexpr int SM_X = SM_W2T + HW * HW;        // chunk features [row][f]
constexpr int SM_T = SM_X + CS * F;           // chunk targets
constexpr int SM_DY = SM_T + CS;              // dLoss/dy per row
constexpr int SM_L = SM_DY + CS;              // squared residual per row
constexpr int SM_A1 = SM_L + CS;              // h1 [row][LDA]
constexpr int SM_A2 = SM_A1 + CS * LDA;       // h2
constexpr int SM_D1 = SM_A2 + CS * LDA;       // gelu'(z1), then dLoss/dz1
constexpr int SM_D2 = SM_D1 + CS * LDA;       // gelu'(z2), then dLoss/dz2
constexpr int SM_FWD_END = SM_D2 + CS * LDA;
constexpr int SM_G = SM_FWD_END;              // gradient, parameter layout
constexpr int SM_P = SM_G + NP + 3;           // master weights
constexpr int SM_M = SM_P + NP + 3;           // Adam first moment
constexpr int SM_V = SM_M + NP + 3;           // Adam second moment
constexpr int SM_MISC = SM_V + NP + 3;        // [0] loss sum
constexpr int SM_TRAIN_END = SM_MISC + 4;
constexpr size_t SMEM_TRAIN = (size_t)SM_TRAIN_END * sizeof(float);
constexpr size_t SMEM_PREDICT = (size_t)SM_FWD_END * sizeof(float);

__device__ __forceinline__ float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ float gelu_fwd(float u, float& d) {
    const float t = tanhf(C_GELU * (u + 0.044715f * u * u * u));
    d = 0.5f * (1.f + t) + 0.5f * u * (1.f - t * t) * C_GELU * (1.f + 3.f * 0.044715f * u * u);
    return 0.5f * u * (1.f + t);
}

// effective weight p from a master value
__device__ __forceinline__ void put_weight(float* sm, int p, float w, int bf16) {
    const float e = bf16 ? round_bf16(w) : w;
    sm[SM_W + p] = e;
    if (p >= OFF_W2 && p < OFF_B2) {
        const int o = (p - OFF_W2) / HW, i = (p - OFF_W2) % HW;
        sm[SM_W2T + i * HW + o] = e;
    }
}

// Forward pass of the rows in sm[SM_X] (rows >= cs are zero).  Leaves h1, h2, gelu'(z1),
// gelu'(z2) in the activation tiles and returns through y the output of row tid >> 2 in the
// lanes with (tid & 3) == 0.
__device__ float forward_chunk(float* sm) {
    const int tid = threadIdx.x;
    // layer 1: thread owns output o for rows r0, r0 + 4, ...
    {
        const int o = tid & (HW - 1);
        float w[F];
#pragma unroll
        for (int f = 0; f < F; ++f) w[f] = sm[SM_W + OFF_W1 + o * F + f];
        const float b = sm[SM_W + OFF_B1 + o];
        for (int r = tid >> 6; r < CS; r += NT / HW) {
            float z = b;
#pragma unroll
            for (int f = 0; f < F; ++f) z = fmaf(w[f], sm[SM_X + r * F + f], z);
            float d;
            sm[SM_A1 + r * LDA + o] = gelu_fwd(z, d);
            sm[SM_D1 + r * LDA + o] = d;
        }
    }
    __syncthreads();
    // layer 2: 4 x 4 register tile, rows ty + 16 j, outputs tx + 16 k
    {
        const int ty = tid >> 4, tx = tid & 15;
        float acc[4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float b = sm[SM_W + OFF_B2 + tx + 16 * k];
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[j][k] = b;
        }
        for (int i = 0; i < HW; ++i) {
            float a[4], w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) a[j] = sm[SM_A1 + (ty + 16 * j) * LDA + i];
#pragma unroll
            for (int k = 0; k < 4; ++k) w[k] = sm[SM_W2T + i * HW + tx + 16 * k];
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[j][k] = fmaf(a[j], w[k], acc[j][k]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int r = ty + 16 * j, o = tx + 16 * k;
                float d;
                sm[SM_A2 + r * LDA + o] = gelu_fwd(acc[j][k], d);
                sm[SM_D2 + r * LDA + o] = d;
            }
    }
    __syncthreads();
    // output: four lanes per row, 16 hidden units each, fixed-order combination
    const int r = tid >> 2, part = tid & 3;
    float y = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) y = fmaf(sm[SM_W + OFF_W3 + part * 16 + k], sm[SM_A2 + r * LDA + part * 16 + k], y);
    y += __shfl_xor_sync(0xffffffffu, y, 1);
    y += __shfl_xor_sync(0xffffffffu, y, 2);
    return y + sm[SM_W + OFF_B3];
}

__global__ void __launch_bounds__(NT, 1)
rm_train_kernel(float* __restrict__ params, float* __restrict__ adam_m, float* __restrict__ adam_v,
                const float* __restrict__ X, const float* __restrict__ T, int64_t n, const int32_t* __restrict__ idx,
                uint64_t data_key, int steps, int batch, int64_t step0, float lr, int bf16, int grad_only,
                float* __restrict__ loss_out, float* __restrict__ grad_out, int* __restrict__ err) {
    extern __shared__ float sm[];
    const int tid = threadIdx.x;
    for (int p = tid; p < NP; p += NT) {
        const float w = params[p];
        sm[SM_P + p] = w;
        sm[SM_M + p] = adam_m[p];
        sm[SM_V + p] = adam_v[p];
        put_weight(sm, p, w, bf16);
    }
    __syncthreads();
    const float inv_b = 1.f / (float)batch;
    const int ty = tid >> 4, tx = tid & 15;
    for (int st = 0; st < steps; ++st) {
        float gW2[4][4] = {};
        float gW1a = 0.f, gW1b = 0.f, gcol = 0.f, gb1 = 0.f, gsc = 0.f;
        for (int c0 = 0; c0 < batch; c0 += CS) {
            const int cs = min(CS, batch - c0);
            // gather the chunk's rows
            for (int e = tid; e < CS * F; e += NT) {
                const int r = e / F, f = e % F;
                float v = 0.f;
                if (r < cs) {
                    const int j = c0 + r;
                    int64_t row;
                    if (grad_only) row = j;
                    else if (idx) row = idx[(int64_t)st * batch + j];
                    else row = (int64_t)(splitmix_at(data_key, (uint64_t)(step0 + st) * (uint64_t)batch + (uint64_t)j) %
                                         (uint64_t)n);
                    if (row < 0 || row >= n) {
                        // reported to the host; the row contributes nothing
                        if (f == 0) {
                            atomicExch(err, 1);
                            sm[SM_T + r] = 0.f;
                        }
                    } else {
                        v = X[row * F + f];
                        if (f == 0) sm[SM_T + r] = T[row];
                    }
                }
                sm[SM_X + e] = v;
            }
            __syncthreads();
            const float y = forward_chunk(sm);
            if ((tid & 3) == 0) {
                const int r = tid >> 2;
                const float res = (r < cs) ? (y - sm[SM_T + r]) : 0.f;
                sm[SM_DY + r] = 2.f * res * inv_b;
                sm[SM_L + r] = res * res;
            }
            __syncthreads();
            // dLoss/dz2 = dy * W3 * gelu'(z2), in place
            {
                const int o = tid & (HW - 1);
                const float w3 = sm[SM_W + OFF_W3 + o];
                for (int r = tid >> 6; r < CS; r += NT / HW) sm[SM_D2 + r * LDA + o] *= sm[SM_DY + r] * w3;
            }
            __syncthreads();
            // gW2 tile (outputs tx + 16 k, inputs ty + 16 j) and dLoss/dh1 tile (rows ty + 16 j,
            // inputs tx + 16 k), then dLoss/dz1 in place of gelu'(z1)
            {
                for (int r = 0; r < CS; ++r) {
                    float dz[4], h[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) dz[k] = sm[SM_D2 + r * LDA + tx + 16 * k];
#pragma unroll
                    for (int j = 0; j < 4; ++j) h[j] = sm[SM_A1 + r * LDA + ty + 16 * j];
#pragma unroll
                    for (int j = 0; j < 4; ++j)
#pragma unroll
                        for (int k = 0; k < 4; ++k) gW2[j][k] = fmaf(dz[k], h[j], gW2[j][k]);
                }
                float dh[4][4] = {};
                for (int o = 0; o < HW; ++o) {
                    float dz[4], w[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) dz[j] = sm[SM_D2 + (ty + 16 * j) * LDA + o];
#pragma unroll
                    for (int k = 0; k < 4; ++k) w[k] = sm[SM_W + OFF_W2 + o * HW + tx + 16 * k];
#pragma unroll
                    for (int j = 0; j < 4; ++j)
#pragma unroll
                        for (int k = 0; k < 4; ++k) dh[j][k] = fmaf(dz[j], w[k], dh[j][k]);
                }
                // column sums: gb2 (threads 0..63), gW3 (64..127), gb3 and the loss (128, 129)
                if (tid < HW) {
                    for (int r = 0; r < CS; ++r) gcol += sm[SM_D2 + r * LDA + tid];
                } else if (tid < 2 * HW) {
                    for (int r = 0; r < CS; ++r) gcol = fmaf(sm[SM_DY + r], sm[SM_A2 + r * LDA + tid - HW], gcol);
                } else if (tid == 2 * HW) {
                    for (int r = 0; r < CS; ++r) gsc += sm[SM_DY + r];
                } else if (tid == 2 * HW + 1) {
                    for (int r = 0; r < CS; ++r) gsc += sm[SM_L + r];
                }
                // dLoss/dz1: this thread's own entries of the gelu'(z1) tile (nobody else reads them here)
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int e = SM_D1 + (ty + 16 * j) * LDA + tx + 16 * k;
                        sm[e] *= dh[j][k];
                    }
            }
            __syncthreads();
            // gW1 (output o, features 2 (tid >> 6) and +1) and gb1
            {
                const int o = tid & (HW - 1), f = 2 * (tid >> 6);
                for (int r = 0; r < CS; ++r) {
                    const float dz = sm[SM_D1 + r * LDA + o];
                    gW1a = fmaf(dz, sm[SM_X + r * F + f], gW1a);
                    gW1b = fmaf(dz, sm[SM_X + r * F + f + 1], gW1b);
                    if (tid < HW) gb1 += dz;
                }
            }
            __syncthreads();
        }
        // gradient to shared memory in parameter layout
        {
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int k = 0; k < 4; ++k) sm[SM_G + OFF_W2 + (tx + 16 * k) * HW + ty + 16 * j] = gW2[j][k];
            const int o = tid & (HW - 1), f = 2 * (tid >> 6);
            sm[SM_G + OFF_W1 + o * F + f] = gW1a;
            sm[SM_G + OFF_W1 + o * F + f + 1] = gW1b;
            if (tid < HW) {
                sm[SM_G + OFF_B1 + tid] = gb1;
                sm[SM_G + OFF_B2 + tid] = gcol;
            } else if (tid < 2 * HW) {
                sm[SM_G + OFF_W3 + tid - HW] = gcol;
            } else if (tid == 2 * HW) {
                sm[SM_G + OFF_B3] = gsc;
            } else if (tid == 2 * HW + 1) {
                sm[SM_MISC] = gsc * inv_b;
            }
        }
        __syncthreads();
        if (grad_only) {
            for (int p = tid; p < NP; p += NT) grad_out[p] = sm[SM_G + p];
            if (tid == 0 && loss_out) loss_out[0] = sm[SM_MISC];
            return;
        }
        if (tid == 0 && loss_out) loss_out[st] = sm[SM_MISC];
        // Adam (Kingma and Ba 2015), bias-corrected
        const float t = (float)(step0 + st + 1);
        const float bc1 = 1.f - powf(BETA1, t), bc2 = 1.f - powf(BETA2, t);
        for (int p = tid; p < NP; p += NT) {
            const float g = sm[SM_G + p];
            const float m = BETA1 * sm[SM_M + p] + (1.f - BETA1) * g;
            const float v = BETA2 * sm[SM_V + p] + (1.f - BETA2) * g * g;
            sm[SM_M + p] = m;
            sm[SM_V + p] = v;
            const float w = sm[SM_P + p] - lr * (m / bc1) / (sqrtf(v / bc2) + ADAM_EPS);
            sm[SM_P + p] = w;
            put_weight(sm, p, w, bf16);
        }
        __syncthreads();
    }
    for (int p = tid; p < NP; p += NT) {
        params[p] = sm[SM_P + p];
        adam_m[p] = sm[SM_M + p];
        adam_v[p] = sm[SM_V + p];
    }
}

__global__ void __launch_bounds__(NT)
rm_predict_kernel(const float* __restrict__ params, int bf16, const float* __restrict__ X, int64_t n,
                  float* __restrict__ Y) {
    extern __shared__ float sm[];
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * CS;
    for (int p = tid; p < NP; p += NT) put_weight(sm, p, params[p], bf16);
    for (int e = tid; e < CS * F; e += NT) {
        const int64_t r = r0 + e / F;
        sm[SM_X + e] = (r < n) ? X[r * F + e % F] : 0.f;
    }
    __syncthreads();
    const float y = forward_chunk(sm);
    const int64_t r = r0 + (tid >> 2);
    if ((tid & 3) == 0 && r < n) Y[r] = y;
}

__global__ void rm_init_kernel(float* __restrict__ params, uint64_t key) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < NP; p += gridDim.x * blockDim.x) {
        float bound = 0.f;
        if (p < OFF_B1) bound = 0.35355339059327373f;                              // 1/sqrt(8)
        else if ((p >= OFF_W2 && p < OFF_B2) || (p >= OFF_W3 && p < OFF_B3)) bound = 0.125f;   // 1/sqrt(64)
        const float u = (float)(splitmix_at(key, (uint64_t)p) >> 40) * 0x1p-24f;
        params[p] = (2.f * u - 1.f) * bound;
    }
}

void check_device(const h2_rankmodel_s* m) {
    int d = -1;
    H2_CUDA(cudaGetDevice(&d));
    if (d != m->device) fail(H2_ERR_INVALID_ARG, "rank model: called with another device current than at creation");
}

void check_dev_ptr(const void* p, const char* what) {
    cudaPointerAttributes a{};
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess ||
        (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        fail(H2_ERR_INVALID_ARG, std::string("rank model: ") + what + " must be a device pointer");
    }
}

void set_smem_attrs() {
    static bool done = false;
    if (done) return;
    H2_CUDA(cudaFuncSetAttribute(rm_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_TRAIN));
    H2_CUDA(cudaFuncSetAttribute(rm_predict_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_PREDICT));
    done = true;
}

}  // namespace

h2_rankmodel_s* rm_create(uint64_t seed, int bf16) {
    auto* m = new h2_rankmodel_s();
    try {
        H2_CUDA(cudaGetDevice(&m->device));
        m->bf16 = bf16 ? 1 : 0;
        m->seed = seed;
        m->params.alloc(NP);
        m->adam_m.alloc(NP);
        m->adam_v.alloc(NP);
        m->grad.alloc(NP);
        m->loss.alloc(1);
        m->err.alloc(1);
        H2_CUDA(cudaMemset(m->err.p, 0, sizeof(int)));
        set_smem_attrs();
        rm_init_kernel<<<(NP + NT - 1) / NT, NT>>>(m->params.p, rng_key(seed, STREAM_MLP_INIT, 0));
        after_launch("rm_init_kernel");
        H2_CUDA(cudaMemset(m->adam_m.p, 0, NP * sizeof(float)));
        H2_CUDA(cudaMemset(m->adam_v.p, 0, NP * sizeof(float)));
        H2_CUDA(cudaDeviceSynchronize());
    } catch (...) {
        delete m;
        throw;
    }
    return m;
}

void rm_free(h2_rankmodel_s* m) { delete m; }

// Reports (and clears) an out-of-range minibatch index seen by an earlier training launch.
void check_err(h2_rankmodel_s* m) {
    int e = 0;
    H2_CUDA(cudaDeviceSynchronize());
    H2_CUDA(cudaMemcpy(&e, m->err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        H2_CUDA(cudaMemset(m->err.p, 0, sizeof(int)));
        fail(H2_ERR_DEVICE_CHECK, "rank model: a training minibatch index was outside [0, n)");
    }
}

void rm_get(h2_rankmodel_s* m, float* p, float* am, float* av, int64_t* step) {
    check_device(m);
    check_err(m);
    if (p) H2_CUDA(cudaMemcpy(p, m->params.p, NP * sizeof(float), cudaMemcpyDeviceToHost));
    if (am) H2_CUDA(cudaMemcpy(am, m->adam_m.p, NP * sizeof(float), cudaMemcpyDeviceToHost));
    if (av) H2_CUDA(cudaMemcpy(av, m->adam_v.p, NP * sizeof(float), cudaMemcpyDeviceToHost));
    if (step) *step = m->step;
}

void rm_set(h2_rankmodel_s* m, const float* p, const float* am, const float* av, int64_t step) {
    check_device(m);
    H2_CUDA(cudaDeviceSynchronize());
    if (p) H2_CUDA(cudaMemcpy(m->params.p, p, NP * sizeof(float), cudaMemcpyHostToDevice));
    if (am) H2_CUDA(cudaMemcpy(m->adam_m.p, am, NP * sizeof(float), cudaMemcpyHostToDevice));
    if (av) H2_CUDA(cudaMemcpy(m->adam_v.p, av, NP * sizeof(float), cudaMemcpyHostToDevice));
    if (step >= 0) m->step = step;
}

namespace {
constexpr char RM_MAGIC[8] = {'H', '2', 'R', 'M', '0', '0', '0', '1'};

struct FileCloser {
    FILE* f;
    ~FileCloser() {
        if (f) fclose(f);
    }
};
}  // namespace

void rm_save(h2_rankmodel_s* m, const char* path) {
    std::vector<float> p(NP), am(NP), av(NP);
    int64_t step = 0;
    rm_get(m, p.data(), am.data(), av.data(), &step);
    FileCloser fc{fopen(path, "wb")};
    if (!fc.f) fail(H2_ERR_INVALID_ARG, std::string("h2_rankmodel_save: cannot open ") + path);
    const int32_t np = NP, bf16 = m->bf16;
    bool ok = fwrite(RM_MAGIC, 1, 8, fc.f) == 8 && fwrite(&np, 4, 1, fc.f) == 1 && fwrite(&bf16, 4, 1, fc.f) == 1 &&
              fwrite(&m->seed, 8, 1, fc.f) == 1 && fwrite(&step, 8, 1, fc.f) == 1 &&
              fwrite(p.data(), 4, NP, fc.f) == (size_t)NP && fwrite(am.data(), 4, NP, fc.f) == (size_t)NP &&
              fwrite(av.data(), 4, NP, fc.f) == (size_t)NP;
    ok = (fclose(fc.f) == 0) && ok;
    fc.f = nullptr;
    if (!ok) fail(H2_ERR_INVALID_ARG, std::string("h2_rankmodel_save: write to ") + path + " failed");
}

h2_rankmodel_s* rm_load(const char* path) {
    FileCloser fc{fopen(path, "rb")};
    if (!fc.f) fail(H2_ERR_INVALID_ARG, std::string("h2_rankmodel_load: cannot open ") + path);
    char magic[8];
    int32_t np = 0, bf16 = 0;
    uint64_t seed = 0;
    int64_t step = 0;
    std::vector<float> p(NP), am(NP), av(NP);
    bool ok = fread(magic, 1, 8, fc.f) == 8 && std::memcmp(magic, RM_MAGIC, 8) == 0 && fread(&np, 4, 1, fc.f) == 1 &&
              np == NP && fread(&bf16, 4, 1, fc.f) == 1 && fread(&seed, 8, 1, fc.f) == 1 &&
              fread(&step, 8, 1, fc.f) == 1 && step >= 0 && fread(p.data(), 4, NP, fc.f) == (size_t)NP &&
              fread(am.data(), 4, NP, fc.f) == (size_t)NP && fread(av.data(), 4, NP, fc.f) == (size_t)NP;
    char extra;
    ok = ok && fread(&extra, 1, 1, fc.f) == 0;
    if (!ok) fail(H2_ERR_INVALID_ARG, std::string("h2_rankmodel_load: ") + path + " is not a rank model file");
    h2_rankmodel_s* m = rm_create(seed, bf16);
    try {
        rm_set(m, p.data(), am.data(), av.data(), step);
    } catch (...) {
        delete m;
        throw;
    }
    return m;
}

void rm_features(const h2_tree_s* t, double kT, double dens, double tol, double* out) {
    const int L = t->L, dim = t->dim;
    auto diam = [&](int l, int b) {
        double s = 0.0;
        for (int d = 0; d < dim; ++d) {
            const double e = t->hi[l][(size_t)b * dim + d] - t->lo[l][(size_t)b * dim + d];
            s += e * e;
        }
        return std::sqrt(s);
    };
    double root = diam(0, 0);
    if (!(root > 0.0)) root = 1.0;
    for (int l = 0; l <= L; ++l) {
        const int nb = 1 << l;
        double dsum = 0.0, ssum = 0.0;
        for (int b = 0; b < nb; ++b) {
            dsum += diam(l, b);
            ssum += (double)t->size[l][b];
        }
        const double dm = dsum / nb, sz = ssum / nb;
        double* o = out + (size_t)l * F;
        o[0] = (double)l / (double)std::max(L, 1);
        o[1] = std::log2(sz) / 20.0;
        o[2] = dm / root;
        o[3] = std::log10(kT) / 4.0;
        o[4] = dens;
        o[5] = std::log10(tol) / 10.0;
        o[6] = std::log10(std::sqrt(kT) / std::max(dm, 1e-300)) / 2.0;
        o[7] = std::log2((double)t->N) / 20.0;
    }
}

void rm_train(h2_rankmodel_s* m, const float* X, const float* T, int64_t n, const int32_t* idx, int steps, int batch,
              float lr, float* loss_out, cudaStream_t s) {
    check_device(m);
    if (n < 1 || steps < 0 || batch < 1 || batch > MAX_BATCH || !(lr > 0.f) || !std::isfinite(lr))
        fail(H2_ERR_INVALID_ARG, "h2_rankmodel_train: need n >= 1, steps >= 0, batch in 1..1024, lr > 0");
    check_dev_ptr(X, "X");
    check_dev_ptr(T, "t");
    if (idx) check_dev_ptr(idx, "idx");
    if (loss_out) check_dev_ptr(loss_out, "loss_out");
    if (steps == 0) return;
    set_smem_attrs();
    rm_train_kernel<<<1, NT, SMEM_TRAIN, s>>>(m->params.p, m->adam_m.p, m->adam_v.p, X, T, n, idx,
                                              rng_key(m->seed, STREAM_MLP_DATA, 0), steps, batch, m->step, lr, m->bf16,
                                              0, loss_out, nullptr, m->err.p);
    after_launch("rm_train_kernel");
    m->step += steps;
}

void rm_loss_grad(h2_rankmodel_s* m, const float* X, const float* T, int64_t n, float* loss, float* grad) {
    check_device(m);
    if (n < 1 || n > MAX_BATCH * 64) fail(H2_ERR_INVALID_ARG, "h2_rankmodel_loss_grad: need 1 <= n <= 65536");
    check_dev_ptr(X, "X");
    check_dev_ptr(T, "t");
    set_smem_attrs();
    rm_train_kernel<<<1, NT, SMEM_TRAIN>>>(m->params.p, m->adam_m.p, m->adam_v.p, X, T, n, nullptr, 0ull, 1, (int)n,
                                           m->step, 1.f, m->bf16, 1, m->loss.p, m->grad.p, m->err.p);
    after_launch("rm_train_kernel");
    H2_CUDA(cudaDeviceSynchronize());
    if (loss) H2_CUDA(cudaMemcpy(loss, m->loss.p, sizeof(float), cudaMemcpyDeviceToHost));
    if (grad) H2_CUDA(cudaMemcpy(grad, m->grad.p, NP * sizeof(float), cudaMemcpyDeviceToHost));
}

void rm_predict(h2_rankmodel_s* m, const float* X, int64_t n, float* Y, cudaStream_t s) {
    check_device(m);
    if (n < 0) fail(H2_ERR_INVALID_ARG, "h2_rankmodel_predict: n < 0");
    if (n == 0) return;
    check_dev_ptr(X, "X");
    check_dev_ptr(Y, "y");
    set_smem_attrs();
    const int64_t grid = (n + CS - 1) / CS;
    if (grid > 0x7fffffff) fail(H2_ERR_INVALID_ARG, "h2_rankmodel_predict: n too large");
    rm_predict_kernel<<<(unsigned)grid, NT, SMEM_PREDICT, s>>>(m->params.p, m->bf16, X, n, Y);
    after_launch("rm_predict_kernel");
}

void rm_q_levels(h2_rankmodel_s* m, const h2_tree_s* t, double kT, double dens, double tol, int pad, int q_max,
                 int32_t* q, float* y_host) {
    check_device(m);
    check_err(m);
    const int L = t->L;
    std::vector<double> f((size_t)(L + 1) * F);
    rm_features(t, kT, dens, tol, f.data());
    std::vector<float> ff(f.begin(), f.end());
    m->feat.reserve(ff.size());
    m->pred.reserve((size_t)L + 1);
    H2_CUDA(cudaMemcpy(m->feat.p, ff.data(), ff.size() * sizeof(float), cudaMemcpyHostToDevice));
    rm_predict(m, m->feat.p, L + 1, m->pred.p, nullptr);
    std::vector<float> y((size_t)L + 1);
    H2_CUDA(cudaMemcpy(y.data(), m->pred.p, y.size() * sizeof(float), cudaMemcpyDeviceToHost));
    q[0] = 0;
    for (int l = 1; l <= L; ++l) {
        const double yl = (double)y[l];
        int v;
        if (!std::isfinite(yl)) v = 0;                              // no prediction: keep q0
        else if (yl > 30.0) v = q_max;
        else {
            int64_t c = (int64_t)std::ceil(std::exp2(yl)) - 1 + pad;
            c = (c + 7) / 8 * 8;
            v = (int)std::min<int64_t>(std::max<int64_t>(c, 8), q_max);
        }
        q[l] = v;
    }
    if (y_host) std::memcpy(y_host, y.data(), y.size() * sizeof(float));
}

}  // namespace h2
