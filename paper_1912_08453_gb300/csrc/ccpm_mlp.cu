// ccpm_mlp.cu -- the constraint-ordering network: a 3-layer perceptron
// (16 -> 64 -> 64 -> 1, ReLU) with BF16 tensor-core forward and backward
// kernels (mma.sync m16n8k16, FP32 accumulate), FP32 master weights and an
// Adam update.  It scores non-local constraints; the pruning pipeline runs
// the best-scored remaining constraint next (every constraint still runs).
//
// Numerics (both here and in the CPU reference the tests compare against):
// inputs X, weights W1/W2 and the hidden activations H1 are rounded to BF16
// before each tensor-core product; products accumulate in FP32; biases, the
// last layer (64 -> 1 dot product), the loss and all gradient reductions
// across the batch are FP32.  The backward products (dW2 = H1^T dZ2,
// dZ1 = dZ2 W2^T, dW1 = X^T dZ1) round their operands (H1, dZ2, W2, X, dZ1)
// to BF16 the same way.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "ccpm_internal.h"

namespace ccpm {

constexpr int IN = CCPM_MLP_IN, HID = CCPM_MLP_HIDDEN;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + IN * HID, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID,
              OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID, NPARAM = OFF_B3 + 1;
static_assert(NPARAM == CCPM_MLP_PARAMS, "parameter layout");
constexpr int ROWS = 64;          // batch rows per CTA
constexpr int THREADS = 128;      // 4 warps

// ---------------------------------------------------------------- mma core

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    uint32_t l = (uint32_t)__bfloat16_as_ushort(lo), h = (uint32_t)__bfloat16_as_ushort(hi);
    return l | (h << 16);
}

// Strided view of a BF16 matrix in shared memory: element (r, c) at
// base[r * rs + c * cs] (a transposed view swaps the strides).
struct View {
    const __nv_bfloat16 *p;
    int rs, cs;
    __device__ __forceinline__ __nv_bfloat16 at(int r, int c) const { return p[r * rs + c * cs]; }
};

// C[M x N] (+)= A[M x K] B[K x N] with all operands in shared memory; the
// CTA's warps share the 16 x 8 output tiles.  C is FP32 with row stride ldc.
__device__ void cta_gemm(View A, View B, float *C, int ldc, int M, int N, int K, bool accumulate) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int g = lane >> 2, tq = lane & 3;
    const int tiles = (M / 16) * (N / 8);
    for (int t = warp; t < tiles; t += nw) {
        const int m0 = (t / (N / 8)) * 16, n0 = (t % (N / 8)) * 8;
        float c[4];
        if (accumulate) {
            c[0] = C[(m0 + g) * ldc + n0 + tq * 2];
            c[1] = C[(m0 + g) * ldc + n0 + tq * 2 + 1];
            c[2] = C[(m0 + g + 8) * ldc + n0 + tq * 2];
            c[3] = C[(m0 + g + 8) * ldc + n0 + tq * 2 + 1];
        } else {
            c[0] = c[1] = c[2] = c[3] = 0.f;
        }
        for (int k0 = 0; k0 < K; k0 += 16) {
            const uint32_t a0 = pack2(A.at(m0 + g, k0 + tq * 2), A.at(m0 + g, k0 + tq * 2 + 1));
            const uint32_t a1 = pack2(A.at(m0 + g + 8, k0 + tq * 2), A.at(m0 + g + 8, k0 + tq * 2 + 1));
            const uint32_t a2 = pack2(A.at(m0 + g, k0 + tq * 2 + 8), A.at(m0 + g, k0 + tq * 2 + 9));
            const uint32_t a3 = pack2(A.at(m0 + g + 8, k0 + tq * 2 + 8), A.at(m0 + g + 8, k0 + tq * 2 + 9));
            const uint32_t b0 = pack2(B.at(k0 + tq * 2, n0 + g), B.at(k0 + tq * 2 + 1, n0 + g));
            const uint32_t b1 = pack2(B.at(k0 + tq * 2 + 8, n0 + g), B.at(k0 + tq * 2 + 9, n0 + g));
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
        C[(m0 + g) * ldc + n0 + tq * 2] = c[0];
        C[(m0 + g) * ldc + n0 + tq * 2 + 1] = c[1];
        C[(m0 + g + 8) * ldc + n0 + tq * 2] = c[2];
        C[(m0 + g + 8) * ldc + n0 + tq * 2 + 1] = c[3];
    }
}

// ------------------------------------------------------------- forward

struct FwdSmem {
    __nv_bfloat16 x[ROWS * IN];
    __nv_bfloat16 w1[IN * HID];
    __nv_bfloat16 w2[HID * HID];
    __nv_bfloat16 h1b[ROWS * HID];
    float z1[ROWS * HID];
    float z2[ROWS * HID];
};

// Forward pass of one 64-row tile: z1 = X W1 + b1, h1 = relu(z1),
// z2 = h1 W2 + b2, h2 = relu(z2), y = h2 . w3 + b3.
__device__ void forward_tile(const float *__restrict__ prm, const float *__restrict__ X, int B, int row0,
                             FwdSmem &S) {
    for (int i = threadIdx.x; i < ROWS * IN; i += blockDim.x) {
        const int r = i / IN;
        S.x[i] = __float2bfloat16_rn(row0 + r < B ? X[(size_t)(row0 + r) * IN + (i % IN)] : 0.f);
    }
    for (int i = threadIdx.x; i < IN * HID; i += blockDim.x) S.w1[i] = __float2bfloat16_rn(prm[OFF_W1 + i]);
    for (int i = threadIdx.x; i < HID * HID; i += blockDim.x) S.w2[i] = __float2bfloat16_rn(prm[OFF_W2 + i]);
    __syncthreads();
    cta_gemm(View{S.x, IN, 1}, View{S.w1, HID, 1}, S.z1, HID, ROWS, HID, IN, false);
    __syncthreads();
    for (int i = threadIdx.x; i < ROWS * HID; i += blockDim.x) {
        const float z = S.z1[i] + prm[OFF_B1 + (i % HID)];
        S.z1[i] = z;
        S.h1b[i] = __float2bfloat16_rn(z > 0.f ? z : 0.f);
    }
    __syncthreads();
    cta_gemm(View{S.h1b, HID, 1}, View{S.w2, HID, 1}, S.z2, HID, ROWS, HID, HID, false);
    __syncthreads();
    for (int i = threadIdx.x; i < ROWS * HID; i += blockDim.x) S.z2[i] += prm[OFF_B2 + (i % HID)];
    __syncthreads();
}

__device__ float out_row(const float *__restrict__ prm, const FwdSmem &S, int r) {
    float y = prm[OFF_B3];
    for (int j = 0; j < HID; j++) {
        const float h = S.z2[r * HID + j];
        y += (h > 0.f ? h : 0.f) * prm[OFF_W3 + j];
    }
    return y;
}

__global__ void __launch_bounds__(THREADS) k_mlp_forward(const float *prm, const float *X, int B, float *Y) {
    extern __shared__ __align__(16) unsigned char smem[];
    FwdSmem &S = *reinterpret_cast<FwdSmem *>(smem);
    for (int row0 = blockIdx.x * ROWS; row0 < B; row0 += gridDim.x * ROWS) {
        forward_tile(prm, X, B, row0, S);
        for (int r = threadIdx.x; r < ROWS; r += blockDim.x)
            if (row0 + r < B) Y[row0 + r] = out_row(prm, S, r);
        __syncthreads();
    }
}

// ------------------------------------------------------------- backward

struct BwdSmem {
    FwdSmem f;
    __nv_bfloat16 dz2b[ROWS * HID];
    __nv_bfloat16 dz1b[ROWS * HID];
    float dz2[ROWS * HID];
    float dz1[ROWS * HID];
    float gw2[HID * HID];
    float gw1[IN * HID];
    float dy[ROWS];
};

// Loss 0.5 * mean((y - t)^2) over the rows idx[0..B): gradients of every
// parameter are added (FP32 atomics) into grad, the summed squared error into
// *sse.  idx may be NULL (rows 0..B-1).
__global__ void __launch_bounds__(THREADS)
k_mlp_backward(const float *prm, const float *X, const float *T, const int32_t *idx, int B, float inv_n,
               float *grad, float *sse) {
    extern __shared__ __align__(16) unsigned char smem[];
    BwdSmem &S = *reinterpret_cast<BwdSmem *>(smem);
    // gather this tile's rows into a dense staging copy of X (in z1 scratch)
    for (int row0 = blockIdx.x * ROWS; row0 < B; row0 += gridDim.x * ROWS) {
        // forward, reading X through idx
        for (int i = threadIdx.x; i < ROWS * IN; i += blockDim.x) {
            const int r = i / IN, row = row0 + r;
            float v = 0.f;
            if (row < B) {
                const int src = idx ? idx[row] : row;
                v = X[(size_t)src * IN + (i % IN)];
            }
            S.f.x[i] = __float2bfloat16_rn(v);
        }
        for (int i = threadIdx.x; i < IN * HID; i += blockDim.x) S.f.w1[i] = __float2bfloat16_rn(prm[OFF_W1 + i]);
        for (int i = threadIdx.x; i < HID * HID; i += blockDim.x) S.f.w2[i] = __float2bfloat16_rn(prm[OFF_W2 + i]);
        __syncthreads();
        cta_gemm(View{S.f.x, IN, 1}, View{S.f.w1, HID, 1}, S.f.z1, HID, ROWS, HID, IN, false);
        __syncthreads();
        for (int i = threadIdx.x; i < ROWS * HID; i += blockDim.x) {
            const float z = S.f.z1[i] + prm[OFF_B1 + (i % HID)];
            S.f.z1[i] = z;
            S.f.h1b[i] = __float2bfloat16_rn(z > 0.f ? z : 0.f);
        }
        __syncthreads();
        cta_gemm(View{S.f.h1b, HID, 1}, View{S.f.w2, HID, 1}, S.f.z2, HID, ROWS, HID, HID, false);
        __syncthreads();
        for (int i = threadIdx.x; i < ROWS * HID; i += blockDim.x) S.f.z2[i] += prm[OFF_B2 + (i % HID)];
        __syncthreads();
        // output layer and dL/dy
        for (int r = threadIdx.x; r < ROWS; r += blockDim.x) {
            const int row = row0 + r;
            float d = 0.f;
            if (row < B) {
                const float y = out_row(prm, S.f, r);
                const int src = idx ? idx[row] : row;
                const float e = y - T[src];
                atomicAdd(sse, e * e);
                d = e * inv_n;
            }
            S.dy[r] = d;
        }
        __syncthreads();
        // w3, b3 and dz2 = dy * w3 * relu'(z2)
        for (int j = threadIdx.x; j < HID; j += blockDim.x) {
            float gw3 = 0.f;
            for (int r = 0; r < ROWS; r++) {
                const float h = S.f.z2[r * HID + j];
                gw3 += S.dy[r] * (h > 0.f ? h : 0.f);
            }
            atomicAdd(&grad[OFF_W3 + j], gw3);
        }
        if (threadIdx.x == 0) {
            float gb3 = 0.f;
            for (int r = 0; r < ROWS; r++) gb3 += S.dy[r];
            atomicAdd(&grad[OFF_B3], gb3);
        }
        for (int i = threadIdx.x; i < ROWS * HID; i += blockDim.x) {
            const int r = i / HID, j = i % HID;
            const float d = S.f.z2[i] > 0.f ? S.dy[r] * prm[OFF_W3 + j] : 0.f;
            S.dz2[i] = d;
            S.dz2b[i] = __float2bfloat16_rn(d);
        }
        __syncthreads();
        // dW2 = h1^T dz2 (64 x 64, K = rows); dz1 = (dz2 W2^T) * relu'(z1)
        cta_gemm(View{S.f.h1b, 1, HID}, View{S.dz2b, HID, 1}, S.gw2, HID, HID, HID, ROWS, false);
        cta_gemm(View{S.dz2b, HID, 1}, View{S.f.w2, 1, HID}, S.dz1, HID, ROWS, HID, HID, false);
        __syncthreads();
        for (int i = threadIdx.x; i < HID * HID; i += blockDim.x) atomicAdd(&grad[OFF_W2 + i], S.gw2[i]);
        for (int j = threadIdx.x; j < HID; j += blockDim.x) {
            float gb2 = 0.f;
            for (int r = 0; r < ROWS; r++) gb2 += S.dz2[r * HID + j];
            atomicAdd(&grad[OFF_B2 + j], gb2);
        }
        for (int i = threadIdx.x; i < ROWS * HID; i += blockDim.x) {
            const float d = S.f.z1[i] > 0.f ? S.dz1[i] : 0.f;
            S.dz1[i] = d;
            S.dz1b[i] = __float2bfloat16_rn(d);
        }
        __syncthreads();
        // dW1 = x^T dz1 (16 x 64, K = rows)
        cta_gemm(View{S.f.x, 1, IN}, View{S.dz1b, HID, 1}, S.gw1, HID, IN, HID, ROWS, false);
        __syncthreads();
        for (int i = threadIdx.x; i < IN * HID; i += blockDim.x) atomicAdd(&grad[OFF_W1 + i], S.gw1[i]);
        for (int j = threadIdx.x; j < HID; j += blockDim.x) {
            float gb1 = 0.f;
            for (int r = 0; r < ROWS; r++) gb1 += S.dz1[r * HID + j];
            atomicAdd(&grad[OFF_B1 + j], gb1);
        }
        __syncthreads();
    }
}

// Adam step on FP32 master weights (bias-corrected), then clear the gradient.
__global__ void k_mlp_adam(float *prm, float *grad, float *m1, float *m2, int step, float lr) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x) {
        const float gi = grad[i];
        m1[i] = b1 * m1[i] + (1.f - b1) * gi;
        m2[i] = b2 * m2[i] + (1.f - b2) * gi * gi;
        prm[i] -= lr * (m1[i] / c1) / (sqrtf(m2[i] / c2) + eps);
        grad[i] = 0.f;
    }
}

// Minibatch row indices from a counter-based hash (SplitMix64 finaliser).
__global__ void k_mlp_sample(int32_t *idx, int batch, int n, uint64_t seed, int step) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < batch; i += gridDim.x * blockDim.x) {
        uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)((int64_t)step * batch + i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        idx[i] = (int32_t)(z % (uint64_t)n);
    }
}

}  // namespace ccpm

using namespace ccpm;

struct ccpm_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    float *prm = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr, *sse = nullptr;
    int adam_step = 0;
    // scratch of the public forward call (pipelines score with their context's own)
    ccpm::MlpScratch own;
    std::mutex mu;               // public forward calls may come from several threads
};

namespace {

size_t fwd_smem() { return sizeof(FwdSmem); }
size_t bwd_smem() { return sizeof(BwdSmem); }

int configure_kernels() {
    // batch workers reach this concurrently: configure once, under a lock
    static std::mutex mu;
    static bool done = false;
    std::lock_guard<std::mutex> lock(mu);
    if (done) return CCPM_OK;
    if (cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem()) != cudaSuccess)
        return CCPM_ECUDA;
    if (cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem()) != cudaSuccess)
        return CCPM_ECUDA;
    done = true;
    return CCPM_OK;
}

// Device scratch for one call (X, targets, outputs); freed by the caller.
struct Scratch {
    float *x = nullptr, *t = nullptr, *y = nullptr;
    int32_t *idx = nullptr;
    ~Scratch() { cudaFree(x); cudaFree(t); cudaFree(y); cudaFree(idx); }
};

int tiles(int B) { return (B + ROWS - 1) / ROWS; }

}  // namespace

namespace ccpm {

void mlp_scratch_free(MlpScratch &sc) {
    cudaFree(sc.dx);
    cudaFree(sc.dy);
    if (sc.hx) cudaFreeHost(sc.hx);
    if (sc.hy) cudaFreeHost(sc.hy);
    sc = MlpScratch{};
}

// Forward pass for the pruning pipeline's ordering decisions (host arrays),
// with the caller's scratch: no lock is held while the GPU works, so batch
// workers that score at the same time do not wait for one another.
int mlp_score(ccpm_mlp *m, int B, const float *host_x, float *host_y, void *stream, MlpScratch &sc, void *wait_ev) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!m || B <= 0) return CCPM_EINVAL;
    if (configure_kernels()) return CCPM_ECUDA;
    if (B > sc.cap) {
        mlp_scratch_free(sc);
        const int cap = std::max(B, 256);
        if (cudaMalloc(&sc.dx, sizeof(float) * (size_t)cap * IN) != cudaSuccess ||
            cudaMalloc(&sc.dy, sizeof(float) * (size_t)cap) != cudaSuccess ||
            cudaMallocHost(&sc.hx, sizeof(float) * (size_t)cap * IN) != cudaSuccess ||
            cudaMallocHost(&sc.hy, sizeof(float) * (size_t)cap) != cudaSuccess) {
            mlp_scratch_free(sc);
            return CCPM_ENOMEM;
        }
        sc.cap = cap;
    }
    std::memcpy(sc.hx, host_x, sizeof(float) * (size_t)B * IN);
    cudaError_t e = cudaMemcpyAsync(sc.dx, sc.hx, sizeof(float) * (size_t)B * IN, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_mlp_forward<<<tiles(B), THREADS, fwd_smem(), s>>>(m->prm, sc.dx, B, sc.dy);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc.hy, sc.dy, sizeof(float) * (size_t)B, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && wait_ev) {
        cudaEvent_t ev = (cudaEvent_t)wait_ev;
        e = cudaEventRecord(ev, s);
        if (e == cudaSuccess)
            while ((e = cudaEventQuery(ev)) == cudaErrorNotReady) std::this_thread::yield();
    } else if (e == cudaSuccess) {
        e = cudaStreamSynchronize(s);
    }
    if (e == cudaSuccess) std::memcpy(host_y, sc.hy, sizeof(float) * (size_t)B);
    return e == cudaSuccess ? CCPM_OK : CCPM_ECUDA;
}

}  // namespace ccpm

extern "C" {

int ccpm_mlp_create(ccpm_ctx_t ctx, uint64_t seed, ccpm_mlp_t *out) {
    if (!ctx || !out) return CCPM_EINVAL;
    *out = nullptr;
    int dev = ctx_device(ctx);
    if (cudaSetDevice(dev) != cudaSuccess) return CCPM_ECUDA;
    ccpm_mlp *m = new (std::nothrow) ccpm_mlp();
    if (!m) return CCPM_ENOMEM;
    m->device = dev;
    m->stream = (cudaStream_t)ctx_stream_ptr(ctx);
    if (cudaMalloc(&m->prm, sizeof(float) * NPARAM) != cudaSuccess ||
        cudaMalloc(&m->grad, sizeof(float) * NPARAM) != cudaSuccess ||
        cudaMalloc(&m->m1, sizeof(float) * NPARAM) != cudaSuccess ||
        cudaMalloc(&m->m2, sizeof(float) * NPARAM) != cudaSuccess ||
        cudaMalloc(&m->sse, sizeof(float)) != cudaSuccess) {
        ccpm_mlp_destroy(m);
        return CCPM_ENOMEM;
    }
    // He-uniform initial weights from a SplitMix64 stream, zero biases
    std::vector<float> p(NPARAM, 0.f);
    uint64_t st = seed;
    auto next = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    auto fill = [&](int off, int count, int fan_in) {
        const double a = std::sqrt(6.0 / fan_in);
        for (int i = 0; i < count; i++) p[(size_t)(off + i)] = (float)((2.0 * next() - 1.0) * a);
    };
    fill(OFF_W1, IN * HID, IN);
    fill(OFF_W2, HID * HID, HID);
    fill(OFF_W3, HID, HID);
    int rc = ccpm_mlp_set_params(m, p.data());
    if (rc) { ccpm_mlp_destroy(m); return rc; }
    *out = m;
    return CCPM_OK;
}

void ccpm_mlp_destroy(ccpm_mlp_t m) {
    if (!m) return;
    cudaSetDevice(m->device);
    cudaFree(m->prm); cudaFree(m->grad); cudaFree(m->m1); cudaFree(m->m2); cudaFree(m->sse);
    ccpm::mlp_scratch_free(m->own);
    delete m;
}

int ccpm_mlp_set_params(ccpm_mlp_t m, const float *host_params) {
    if (!m || !host_params) return CCPM_EINVAL;
    if (cudaSetDevice(m->device) != cudaSuccess) return CCPM_ECUDA;
    cudaError_t e = cudaMemcpyAsync(m->prm, host_params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->grad, 0, sizeof(float) * NPARAM, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->m1, 0, sizeof(float) * NPARAM, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->m2, 0, sizeof(float) * NPARAM, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    m->adam_step = 0;
    return e == cudaSuccess ? CCPM_OK : CCPM_ECUDA;
}

int ccpm_mlp_get_params(ccpm_mlp_t m, float *host_params) {
    if (!m || !host_params) return CCPM_EINVAL;
    if (cudaSetDevice(m->device) != cudaSuccess) return CCPM_ECUDA;
    cudaError_t e = cudaMemcpyAsync(host_params, m->prm, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? CCPM_OK : CCPM_ECUDA;
}

int ccpm_mlp_forward(ccpm_mlp_t m, int B, const float *host_x, float *host_y) {
    if (!m || B <= 0 || !host_x || !host_y) return CCPM_EINVAL;
    if (cudaSetDevice(m->device) != cudaSuccess) return CCPM_ECUDA;
    std::lock_guard<std::mutex> lock(m->mu);
    return mlp_score(m, B, host_x, host_y, (void *)m->stream, m->own);
}

int ccpm_mlp_gradient(ccpm_mlp_t m, int B, const float *host_x, const float *host_t, float *host_grad,
                      float *loss) {
    if (!m || B <= 0 || !host_x || !host_t || !host_grad) return CCPM_EINVAL;
    if (cudaSetDevice(m->device) != cudaSuccess) return CCPM_ECUDA;
    if (configure_kernels()) return CCPM_ECUDA;
    Scratch sc;
    if (cudaMalloc(&sc.x, sizeof(float) * (size_t)B * IN) != cudaSuccess ||
        cudaMalloc(&sc.t, sizeof(float) * (size_t)B) != cudaSuccess)
        return CCPM_ENOMEM;
    cudaStream_t s = m->stream;
    cudaError_t e = cudaMemcpyAsync(sc.x, host_x, sizeof(float) * (size_t)B * IN, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc.t, host_t, sizeof(float) * (size_t)B, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->grad, 0, sizeof(float) * NPARAM, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->sse, 0, sizeof(float), s);
    if (e == cudaSuccess) {
        k_mlp_backward<<<tiles(B), THREADS, bwd_smem(), s>>>(m->prm, sc.x, sc.t, nullptr, B, 1.f / (float)B, m->grad,
                                                              m->sse);
        e = cudaGetLastError();
    }
    float sse = 0.f;
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_grad, m->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sse, m->sse, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->grad, 0, sizeof(float) * NPARAM, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (loss) *loss = 0.5f * sse / (float)B;
    return e == cudaSuccess ? CCPM_OK : CCPM_ECUDA;
}

int ccpm_mlp_train(ccpm_mlp_t m, int N, const float *host_x, const float *host_t, int steps, int batch, float lr,
                   uint64_t seed, float *final_loss) {
    if (!m || N <= 0 || !host_x || !host_t || steps < 0 || batch <= 0) return CCPM_EINVAL;
    if (cudaSetDevice(m->device) != cudaSuccess) return CCPM_ECUDA;
    if (configure_kernels()) return CCPM_ECUDA;
    Scratch sc;
    if (cudaMalloc(&sc.x, sizeof(float) * (size_t)N * IN) != cudaSuccess ||
        cudaMalloc(&sc.t, sizeof(float) * (size_t)N) != cudaSuccess ||
        cudaMalloc(&sc.idx, sizeof(int32_t) * (size_t)batch) != cudaSuccess)
        return CCPM_ENOMEM;
    cudaStream_t s = m->stream;
    cudaError_t e = cudaMemcpyAsync(sc.x, host_x, sizeof(float) * (size_t)N * IN, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc.t, host_t, sizeof(float) * (size_t)N, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->grad, 0, sizeof(float) * NPARAM, s);
    for (int it = 0; it < steps && e == cudaSuccess; it++) {
        e = cudaMemsetAsync(m->sse, 0, sizeof(float), s);
        if (e != cudaSuccess) break;
        k_mlp_sample<<<(batch + 255) / 256, 256, 0, s>>>(sc.idx, batch, N, seed, it);
        k_mlp_backward<<<tiles(batch), THREADS, bwd_smem(), s>>>(m->prm, sc.x, sc.t, sc.idx, batch,
                                                                  1.f / (float)batch, m->grad, m->sse);
        m->adam_step++;
        k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(m->prm, m->grad, m->m1, m->m2, m->adam_step, lr);
        e = cudaGetLastError();
    }
    float sse = 0.f;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sse, m->sse, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (final_loss) *final_loss = 0.5f * sse / (float)batch;
    return e == cudaSuccess ? CCPM_OK : CCPM_ECUDA;
}

}  // extern "C"
