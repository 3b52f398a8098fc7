// Selector network of the learned form: forward pass, loss gradient and Adam
// update, FP32 arithmetic on bfloat16 weights.
//
// The paper fixes one truncation number for the whole tree (Sec. 5 names
// "variable truncation number" among the optimisations it left out); the
// learned form picks one per level.  Network (weights W_k (out x in), row-major,
// stored as bfloat16; biases FP32):
//   h1 = relu(W1 x + b1) 12 -> 64,  h2 = relu(W2 h1 + b2) 64 -> 64,
//   h3 = relu(W3 h2 + b3) 64 -> 64, z = W4 h3 + b4 64 -> 21
// z[0:17] score p = 4 .. 20, z[17:21] score the leaf caps 16, 32, 64, 128.
// Loss: mean cross-entropy of the labelled p rows plus mean cross-entropy of the
// labelled leaf rows; gradients by the chain rule through the same layers.
// The network is tiny (10,304 weights): one block of 64 threads per 64 rows,
// weights and activations in shared memory, FP32 atomics to combine blocks.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "lhv_internal.cuh"

namespace lhv {

namespace {

constexpr int IN = LHV_MLP_IN, HID = LHV_MLP_HIDDEN, OUT = LHV_MLP_OUT, NP = LHV_MLP_NP;
constexpr int ROWS = 64;        // rows per block
constexpr int THREADS = 64;
// per layer k = 0..3: input / output widths, offsets of W_k and b_k, and the
// (odd, bank-conflict-free) row stride of W_k in shared memory
__host__ __device__ constexpr int din(int k) { return k == 0 ? IN : HID; }
__host__ __device__ constexpr int dout(int k) { return k == 3 ? OUT : HID; }
__host__ __device__ constexpr int w_off(int k) { return k == 0 ? 0 : HID * IN + (k - 1) * HID * HID; }
__host__ __device__ constexpr int b_off(int k) { return k * HID; }
__host__ __device__ constexpr int ldw(int k) { return din(k) + 1; }
__host__ __device__ constexpr int sw_off(int k) { return k == 0 ? 0 : HID * (IN + 1) + (k - 1) * HID * (HID + 1); }
constexpr int SW_TOTAL = HID * (IN + 1) + 2 * HID * (HID + 1) + OUT * (HID + 1);
constexpr int LDA = HID + 1;

struct Smem {
    float w[SW_TOTAL];
    float b[LHV_MLP_NB];
    float act[4][ROWS][LDA];  // act[0]: input, act[k]: output of layer k (pre-activation for k = 1..3)
    float z[ROWS][OUT + 1];
};

__device__ void stage_weights(Smem& s, const __nv_bfloat16* __restrict__ W, const float* __restrict__ b) {
    for (int k = 0; k < 4; ++k)
        for (int e = threadIdx.x; e < dout(k) * din(k); e += THREADS) {
            const int o = e / din(k), i = e - o * din(k);
            s.w[sw_off(k) + o * ldw(k) + i] = __bfloat162float(W[w_off(k) + e]);
        }
    for (int e = threadIdx.x; e < LHV_MLP_NB; e += THREADS) s.b[e] = b[e];
}

// rows r0 .. r0 + nr - 1: act[0] <- X, act[1..3] <- pre-activations, z <- logits
__device__ void forward_rows(Smem& s, const float* __restrict__ X, int64_t r0, int nr) {
    for (int e = threadIdx.x; e < ROWS * IN; e += THREADS) {
        const int r = e / IN, i = e - r * IN;
        s.act[0][r][i] = r < nr ? X[(r0 + r) * IN + i] : 0.0f;
    }
    __syncthreads();
    for (int k = 0; k < 4; ++k) {
        const int o = threadIdx.x;
        if (o < dout(k)) {
            const float* w = s.w + sw_off(k) + o * ldw(k);
            const float bias = s.b[b_off(k) + o];
            for (int r = 0; r < nr; ++r) {
                float acc = bias;
                for (int i = 0; i < din(k); ++i) {
                    const float a = s.act[k][r][i];
                    acc = fmaf(w[i], k == 0 ? a : fmaxf(a, 0.0f), acc);  // relu of the previous pre-activation
                }
                if (k < 3) s.act[k + 1][r][o] = acc;
                else s.z[r][o] = acc;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(THREADS) k_mlp_forward(int rows, const float* __restrict__ X,
                                                         const __nv_bfloat16* __restrict__ W,
                                                         const float* __restrict__ b, float* __restrict__ Z) {
    extern __shared__ __align__(16) unsigned char raw[];
    Smem& s = *reinterpret_cast<Smem*>(raw);
    stage_weights(s, W, b);
    __syncthreads();
    for (int64_t r0 = (int64_t)blockIdx.x * ROWS; r0 < rows; r0 += (int64_t)gridDim.x * ROWS) {
        const int nr = (int)(rows - r0 < ROWS ? rows - r0 : ROWS);
        forward_rows(s, X, r0, nr);
        for (int e = threadIdx.x; e < nr * OUT; e += THREADS) {
            const int r = e / OUT, o = e - r * OUT;
            Z[(r0 + r) * OUT + o] = s.z[r][o];
        }
        __syncthreads();
    }
}

__global__ void k_mlp_count(int rows, const int* __restrict__ yp, const int* __restrict__ yl, int* __restrict__ cnt) {
    int a = 0, c = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
        a += yp[r] >= 0;
        c += yl[r] >= 0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd(cnt, a);
        if (c) atomicAdd(cnt + 1, c);
    }
}

// softmax cross-entropy of z[lo, hi) against label y; writes dz = (softmax - onehot) * scale
__device__ float xent(const float* z, float* dz, int lo, int hi, int y, float scale) {
    float mx = -INFINITY;
    for (int o = lo; o < hi; ++o) mx = fmaxf(mx, z[o]);
    float sum = 0.0f;
    for (int o = lo; o < hi; ++o) sum += expf(z[o] - mx);
    for (int o = lo; o < hi; ++o) dz[o] = (expf(z[o] - mx) / sum - (o - lo == y ? 1.0f : 0.0f)) * scale;
    return (logf(sum) + mx - z[lo + y]) * scale;
}

__global__ void __launch_bounds__(THREADS) k_mlp_grad(int rows, const float* __restrict__ X, const int* __restrict__ yp,
                                                      const int* __restrict__ yl, const __nv_bfloat16* __restrict__ W,
                                                      const float* __restrict__ b, const int* __restrict__ cnt,
                                                      float* __restrict__ gW, float* __restrict__ gb,
                                                      float* __restrict__ loss) {
    extern __shared__ __align__(16) unsigned char raw[];
    Smem& s = *reinterpret_cast<Smem*>(raw);
    __shared__ float d[2][ROWS][LDA];  // the gradient flowing back, two layers at a time
    stage_weights(s, W, b);
    __syncthreads();
    const float sp = cnt[0] > 0 ? 1.0f / cnt[0] : 0.0f, sl = cnt[1] > 0 ? 1.0f / cnt[1] : 0.0f;
    for (int64_t r0 = (int64_t)blockIdx.x * ROWS; r0 < rows; r0 += (int64_t)gridDim.x * ROWS) {
        const int nr = (int)(rows - r0 < ROWS ? rows - r0 : ROWS);
        forward_rows(s, X, r0, nr);
        // dz and the loss, one row per thread
        float part = 0.0f;
        {
            const int r = threadIdx.x;
            float* dz = d[0][r];
            for (int o = 0; o < OUT; ++o) dz[o] = 0.0f;
            if (r < nr) {
                const int a = yp[r0 + r], c = yl[r0 + r];
                if (a >= 0) part += xent(s.z[r], dz, 0, NP, a, sp);
                if (c >= 0) part += xent(s.z[r], dz, NP, OUT, c, sl);
            }
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        if ((threadIdx.x & 31) == 0 && part != 0.0f) atomicAdd(loss, part);
        __syncthreads();
        int cur = 0;
        for (int k = 3; k >= 0; --k) {
            // gW_k[o][i] = sum_r d[r][o] in_k[r][i],  gb_k[o] = sum_r d[r][o]
            for (int e = threadIdx.x; e < dout(k) * din(k); e += THREADS) {
                const int o = e / din(k), i = e - o * din(k);
                float acc = 0.0f;
                for (int r = 0; r < nr; ++r) {
                    const float a = s.act[k][r][i];
                    acc = fmaf(d[cur][r][o], k == 0 ? a : fmaxf(a, 0.0f), acc);
                }
                atomicAdd(gW + w_off(k) + e, acc);
            }
            if (threadIdx.x < dout(k)) {
                float acc = 0.0f;
                for (int r = 0; r < nr; ++r) acc += d[cur][r][threadIdx.x];
                atomicAdd(gb + b_off(k) + threadIdx.x, acc);
            }
            if (k > 0) {
                // d_{k-1}[r][i] = (sum_o d[r][o] W_k[o][i]) * [pre_k[r][i] > 0]
                const int i = threadIdx.x;
                if (i < din(k))
                    for (int r = 0; r < nr; ++r) {
                        float acc = 0.0f;
                        for (int o = 0; o < dout(k); ++o) acc = fmaf(d[cur][r][o], s.w[sw_off(k) + o * ldw(k) + i], acc);
                        d[cur ^ 1][r][i] = s.act[k][r][i] > 0.0f ? acc : 0.0f;
                    }
            }
            __syncthreads();
            cur ^= 1;
        }
    }
}

// Adam (Kingma & Ba 2015) on the FP32 master weights, then their bfloat16 copy.
__global__ void k_mlp_adam(float* __restrict__ W32, __nv_bfloat16* __restrict__ W, const float* __restrict__ gW,
                           float* __restrict__ mW, float* __restrict__ vW, float* __restrict__ b,
                           const float* __restrict__ gb, float* __restrict__ mb, float* __restrict__ vb, float c1,
                           float c2, float lr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    if (i < LHV_MLP_NW) {
        const float g = gW[i];
        const float m = b1 * mW[i] + (1.0f - b1) * g;
        const float v = b2 * vW[i] + (1.0f - b2) * g * g;
        mW[i] = m;
        vW[i] = v;
        const float w = W32[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
        W32[i] = w;
        W[i] = __float2bfloat16_rn(w);
    } else if (i < LHV_MLP_NW + LHV_MLP_NB) {
        const int j = i - LHV_MLP_NW;
        const float g = gb[j];
        const float m = b1 * mb[j] + (1.0f - b1) * g;
        const float v = b2 * vb[j] + (1.0f - b2) * g * g;
        mb[j] = m;
        vb[j] = v;
        b[j] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

int blocks_for(int rows) { return std::max(1, std::min((rows + ROWS - 1) / ROWS, 152 * 4)); }

}  // namespace

size_t mlp_smem_bytes() { return sizeof(Smem); }

cudaError_t mlp_forward(cudaStream_t s, int rows, const float* X, const uint16_t* W, const float* b, float* Z) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
    if (e != cudaSuccess) return e;
    k_mlp_forward<<<blocks_for(rows), THREADS, sizeof(Smem), s>>>(rows, X, reinterpret_cast<const __nv_bfloat16*>(W),
                                                                  b, Z);
    return cudaGetLastError();
}

cudaError_t mlp_grad(cudaStream_t s, int rows, const float* X, const int* yp, const int* yl, const uint16_t* W,
                     const float* b, float* gW, float* gb, float* loss, int* cnt) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(gW, 0, LHV_MLP_NW * sizeof(float), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(gb, 0, LHV_MLP_NB * sizeof(float), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(loss, 0, sizeof(float), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(cnt, 0, 2 * sizeof(int), s)) != cudaSuccess) return e;
    k_mlp_count<<<std::max(1, std::min((rows + 255) / 256, 152)), 256, 0, s>>>(rows, yp, yl, cnt);
    k_mlp_grad<<<blocks_for(rows), THREADS, sizeof(Smem), s>>>(rows, X, yp, yl,
                                                               reinterpret_cast<const __nv_bfloat16*>(W), b, cnt, gW,
                                                               gb, loss);
    return cudaGetLastError();
}

cudaError_t mlp_adam(cudaStream_t s, float* W32, uint16_t* W, const float* gW, float* mW, float* vW, float* b,
                     const float* gb, float* mb, float* vb, int t, float lr) {
    const float c1 = 1.0f - powf(0.9f, (float)t), c2 = 1.0f - powf(0.999f, (float)t);
    const int n = LHV_MLP_NW + LHV_MLP_NB;
    k_mlp_adam<<<(n + 255) / 256, 256, 0, s>>>(W32, reinterpret_cast<__nv_bfloat16*>(W), gW, mW, vW, b, gb, mb, vb,
                                               c1, c2, lr);
    return cudaGetLastError();
}

}  // namespace lhv
