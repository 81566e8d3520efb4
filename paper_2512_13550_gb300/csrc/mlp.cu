// Learned starting guess: a 3-layer perceptron (FP32) with hand-written forward, back-propagation
// and Adam kernels. The paper has no learned component (it notes that its Python implementation
// suits machine-learning workflows); the network maps per-pair features to the converged
// occupation angle of the pair, trained on solutions the method itself produces.
//
// Network: x (F) -> relu(W1 x + b1) (H) -> relu(W2 h1 + b2) (H) -> W3 h2 + b3 (O); loss = mean
// over the batch of sum_o (y - t)^2. Parameters packed as W1 [H][F], b1 [H], W2 [H][H], b2 [H],
// W3 [O][H], b3 [O]. Work buffer (floats): Z1 [B][H], Z2 [B][H], Y [B][O], dZ2 [B][H], dZ1 [B][H],
// dY [B][O].
#include <cuda_bf16.h>

#include "internal.h"

namespace {

// C(m, n) = sum_k opA(m, k) B(k, n) (+ bias[n]) (* (mask(m, n) > 0)); opA applies relu when
// a_relu is set. Strided operands, 64 x 64 output tile per CTA, 4 x 4 outputs per thread.
struct Gemm32 {
    int M = 0, N = 0, K = 0;
    const float* A = nullptr; long long sAm = 0, sAk = 0; int a_relu = 0;
    const float* B = nullptr; long long sBk = 0, sBn = 0; int b_relu = 0;
    float* C = nullptr; long long sCm = 0, sCn = 0;
    const float* bias = nullptr;                           // [N] or null
    const float* mask = nullptr; long long sMm = 0, sMn = 0;  // or null
};

Gemm32 mk(int M, int N, int K, const float* A, long long sAm, long long sAk, int a_relu, const float* B,
          long long sBk, long long sBn, int b_relu, float* C, long long sCm, long long sCn) {
    Gemm32 g;
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.sAm = sAm; g.sAk = sAk; g.a_relu = a_relu;
    g.B = B; g.sBk = sBk; g.sBn = sBn; g.b_relu = b_relu;
    g.C = C; g.sCm = sCm; g.sCn = sCn;
    return g;
}

__global__ void __launch_bounds__(256) k_gemm32(Gemm32 g) {
    __shared__ float As[16][65];
    __shared__ float Bs[16][65];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int kt = 0; kt < g.K; kt += 16) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            int e = tid + 256 * l;
            int mm = e % 64, kk = e / 64;
            int m = m0 + mm, k = kt + kk;
            float a = (m < g.M && k < g.K) ? g.A[m * g.sAm + k * g.sAk] : 0.f;
            As[kk][mm] = g.a_relu ? fmaxf(a, 0.f) : a;
            int nn = e % 64, kb = e / 64;
            int n = n0 + nn, kq = kt + kb;
            float b = (n < g.N && kq < g.K) ? g.B[kq * g.sBk + n * g.sBn] : 0.f;
            Bs[kb][nn] = g.b_relu ? fmaxf(b, 0.f) : b;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int m = m0 + ty + 16 * i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int n = n0 + tx + 16 * j;
            if (n >= g.N) continue;
            float v = acc[i][j];
            if (g.bias) v += g.bias[n];
            if (g.mask && !(g.mask[m * g.sMm + n * g.sMn] > 0.f)) v = 0.f;
            g.C[m * g.sCm + n * g.sCn] = v;
        }
    }
}

int gemm32(const Gemm32& g, cudaStream_t st) {
    dim3 grid((g.N + 63) / 64, (g.M + 63) / 64);
    k_gemm32<<<grid, 256, 0, st>>>(g);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

// out[n] = sum_m A[m][n] (column sums, one warp per column, fixed order)
__global__ void k_colsum(const float* A, int M, int N, float* out) {
    int n = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (n >= N) return;
    float s = 0.f;
    for (int m = lane; m < M; m += 32) s += A[(long long)m * N + n];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[n] = s;
}

// dY = 2 (Y - T) / B and the loss sum (Y - T)^2 / B (single block, fixed reduction order)
__global__ void k_mse(const float* Y, const float* T, int n, int Bn, float* dY, float* loss) {
    __shared__ float red[1024];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        float r = Y[i] - T[i];
        dY[i] = 2.f * r / Bn;
        s += r * r;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) *loss = red[0] / Bn;
}

// Adam with decoupled weight decay (Loshchilov & Hutter, "Decoupled Weight Decay Regularization",
// ICLR 2019): theta -= lr (mhat / (sqrt(vhat) + eps) + wd theta).
__global__ void k_adam32(long long P, float* th, const float* g, float* m, float* v, float c1, float c2, float lr,
                         float b1, float b2, float eps, float wd) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= P) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * th[i]);
}

struct MlpLayout {
    const float *W1, *b1, *W2, *b2, *W3, *b3;
    float *Z1, *Z2, *Y, *dZ2, *dZ1, *dY;
};

MlpLayout layout(const float* th, float* work, int B, int F, int H, int O) {
    MlpLayout L;
    L.W1 = th; L.b1 = L.W1 + (long long)H * F; L.W2 = L.b1 + H; L.b2 = L.W2 + (long long)H * H;
    L.W3 = L.b2 + H; L.b3 = L.W3 + (long long)O * H;
    L.Z1 = work; L.Z2 = L.Z1 + (long long)B * H; L.Y = L.Z2 + (long long)B * H;
    L.dZ2 = L.Y + (long long)B * O; L.dZ1 = L.dZ2 + (long long)B * H; L.dY = L.dZ1 + (long long)B * H;
    return L;
}

int mlp_forward(const MlpLayout& L, const float* X, int B, int F, int H, int O, cudaStream_t st) {
    Gemm32 g = mk(B, H, F, X, F, 1, 0, L.W1, 1, F, 0, L.Z1, H, 1);  // Z1 = X W1^T + b1
    g.bias = L.b1;
    NOF_TRY(gemm32(g, st));
    g = mk(B, H, H, L.Z1, H, 1, 1, L.W2, 1, H, 0, L.Z2, H, 1);         // Z2 = relu(Z1) W2^T + b2
    g.bias = L.b2;
    NOF_TRY(gemm32(g, st));
    g = mk(B, O, H, L.Z2, H, 1, 1, L.W3, 1, H, 0, L.Y, O, 1);          // Y = relu(Z2) W3^T + b3
    g.bias = L.b3;
    return gemm32(g, st);
}

bool bad_sizes(int B, int F, int H, int O) { return B <= 0 || F <= 0 || H <= 0 || O <= 0; }

// ---- BF16 inference on the tensor cores ---------------------------------------------------------
// One layer Y = act(X W^T + b): X [B][K] FP32 activations (rounded to BF16 as they are loaded),
// W [N][K] BF16 (the converted parameters), b [N] FP32, FP32 accumulation. One warp per 16 x 8
// output tile, mma.sync m16n8k16 over K in steps of 16; rows >= B, columns >= N and K >= Kdim are
// zero-filled on load and not stored.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (low 16 bits) = lo
    return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t load_bf16x2(const __nv_bfloat16* W, long long ld, int n, int k, int N, int K) {
    const unsigned short lo = (n < N && k < K) ? __bfloat16_as_ushort(W[(long long)n * ld + k]) : 0;
    const unsigned short hi = (n < N && k + 1 < K) ? __bfloat16_as_ushort(W[(long long)n * ld + k + 1]) : 0;
    return (uint32_t)lo | ((uint32_t)hi << 16);
}
__global__ void __launch_bounds__(32) k_layer_bf16(const float* X, int B, int K, const __nv_bfloat16* W,
                                                   const float* bias, int N, int relu, float* Y) {
    const int lane = threadIdx.x, grp = lane >> 2, tig = lane & 3;
    const int m0 = blockIdx.x * 16, n0 = blockIdx.y * 8;
    auto xa = [&](int r, int k) { return (r < B && k < K) ? X[(long long)r * K + k] : 0.f; };
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < K; k0 += 16) {
        const int ka = k0 + 2 * tig;
        const uint32_t a0 = pack_bf16x2(xa(m0 + grp, ka), xa(m0 + grp, ka + 1));
        const uint32_t a1 = pack_bf16x2(xa(m0 + grp + 8, ka), xa(m0 + grp + 8, ka + 1));
        const uint32_t a2 = pack_bf16x2(xa(m0 + grp, ka + 8), xa(m0 + grp, ka + 9));
        const uint32_t a3 = pack_bf16x2(xa(m0 + grp + 8, ka + 8), xa(m0 + grp + 8, ka + 9));
        const uint32_t b0 = load_bf16x2(W, K, n0 + grp, ka, N, K);
        const uint32_t b1 = load_bf16x2(W, K, n0 + grp, ka + 8, N, K);
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
    // d0, d1: row grp, columns 2 tig, 2 tig + 1; d2, d3: row grp + 8
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = m0 + grp + (i >= 2 ? 8 : 0), c = n0 + 2 * tig + (i & 1);
        if (r < B && c < N) {
            float v = d[i] + bias[c];
            if (relu) v = fmaxf(v, 0.f);
            Y[(long long)r * N + c] = v;
        }
    }
}
__global__ void k_to_bf16(const float* a, long long n, __nv_bfloat16* out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16_rn(a[i]);
}

}  // namespace

extern "C" {

long long nof_mlp_param_count(int F, int H, int O) {
    return (long long)H * F + H + (long long)H * H + H + (long long)O * H + O;
}

long long nof_mlp_work_size(int B, int H, int O) { return 4ll * B * H + 2ll * B * O; }

int nof_mlp_forward(int B, int F, int H, int O, const float* theta, const float* X, float* Y, float* work,
                    void* stream) {
    if (bad_sizes(B, F, H, O) || !theta || !X || !Y || !work) {
        nof_set_error("nof_mlp_forward: bad sizes or null pointer");
        return NOF_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    MlpLayout L = layout(theta, work, B, F, H, O);
    NOF_TRY(mlp_forward(L, X, B, F, H, O, st));
    NOF_CUDA(cudaMemcpyAsync(Y, L.Y, sizeof(float) * B * O, cudaMemcpyDeviceToDevice, st));
    return NOF_OK;
}

int nof_mlp_loss_grad(int B, int F, int H, int O, const float* theta, const float* X, const float* T,
                      float* loss, float* grad, float* work, void* stream) {
    if (bad_sizes(B, F, H, O) || !theta || !X || !T || !grad || !work) {
        nof_set_error("nof_mlp_loss_grad: bad sizes or null pointer");
        return NOF_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    MlpLayout L = layout(theta, work, B, F, H, O);
    NOF_TRY(mlp_forward(L, X, B, F, H, O, st));
    k_mse<<<1, 1024, 0, st>>>(L.Y, T, B * O, B, L.dY, loss);
    NOF_LAUNCH_CHECK();
    float* gW1 = grad;
    float* gb1 = gW1 + (long long)H * F;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + (long long)H * H;
    float* gW3 = gb2 + H;
    float* gb3 = gW3 + (long long)O * H;
    // gW3 = dY^T relu(Z2), gb3 = colsum(dY)
    NOF_TRY(gemm32(mk(O, H, B, L.dY, 1, O, 0, L.Z2, H, 1, 1, gW3, H, 1), st));
    k_colsum<<<(unsigned)((O * 32 + 255) / 256), 256, 0, st>>>(L.dY, B, O, gb3);
    NOF_LAUNCH_CHECK();
    // dZ2 = (dY W3) * (Z2 > 0)
    Gemm32 g = mk(B, H, O, L.dY, O, 1, 0, L.W3, H, 1, 0, L.dZ2, H, 1);
    g.mask = L.Z2; g.sMm = H; g.sMn = 1;
    NOF_TRY(gemm32(g, st));
    // gW2 = dZ2^T relu(Z1), gb2 = colsum(dZ2)
    NOF_TRY(gemm32(mk(H, H, B, L.dZ2, 1, H, 0, L.Z1, H, 1, 1, gW2, H, 1), st));
    k_colsum<<<(unsigned)((H * 32 + 255) / 256), 256, 0, st>>>(L.dZ2, B, H, gb2);
    NOF_LAUNCH_CHECK();
    // dZ1 = (dZ2 W2) * (Z1 > 0)
    g = mk(B, H, H, L.dZ2, H, 1, 0, L.W2, H, 1, 0, L.dZ1, H, 1);
    g.mask = L.Z1; g.sMm = H; g.sMn = 1;
    NOF_TRY(gemm32(g, st));
    // gW1 = dZ1^T X, gb1 = colsum(dZ1)
    NOF_TRY(gemm32(mk(H, F, B, L.dZ1, 1, H, 0, X, F, 1, 0, gW1, F, 1), st));
    k_colsum<<<(unsigned)((H * 32 + 255) / 256), 256, 0, st>>>(L.dZ1, B, H, gb1);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

int nof_mlp_to_bf16(long long P, const float* theta, void* theta_bf16, void* stream) {
    if (P <= 0 || !theta || !theta_bf16) {
        nof_set_error("nof_mlp_to_bf16: bad arguments");
        return NOF_EINVAL;
    }
    k_to_bf16<<<(unsigned)((P + 255) / 256), 256, 0, (cudaStream_t)stream>>>(theta, P, (__nv_bfloat16*)theta_bf16);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

int nof_mlp_forward_bf16(int B, int F, int H, int O, const void* theta_bf16, const float* theta, const float* X,
                         float* Y, float* work, void* stream) {
    if (bad_sizes(B, F, H, O) || !theta_bf16 || !theta || !X || !Y || !work) {
        nof_set_error("nof_mlp_forward_bf16: bad sizes or null pointer");
        return NOF_EINVAL;
    }
    if ((long long)(B + 15) / 16 > 2147483647LL || (H + 7) / 8 > 65535 || (O + 7) / 8 > 65535) {
        nof_set_error("nof_mlp_forward_bf16: sizes beyond the launch grid");
        return NOF_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const __nv_bfloat16* Wb = (const __nv_bfloat16*)theta_bf16;
    // parameter offsets of the packed layout (the biases are read in FP32)
    const long long oW1 = 0, ob1 = (long long)H * F, oW2 = ob1 + H, ob2 = oW2 + (long long)H * H, oW3 = ob2 + H,
                    ob3 = oW3 + (long long)O * H;
    float* Z1 = work;
    float* Z2 = work + (long long)B * H;
    const unsigned gm = (unsigned)((B + 15) / 16);
    k_layer_bf16<<<dim3(gm, (H + 7) / 8), 32, 0, st>>>(X, B, F, Wb + oW1, theta + ob1, H, 1, Z1);
    NOF_LAUNCH_CHECK();
    k_layer_bf16<<<dim3(gm, (H + 7) / 8), 32, 0, st>>>(Z1, B, H, Wb + oW2, theta + ob2, H, 1, Z2);
    NOF_LAUNCH_CHECK();
    k_layer_bf16<<<dim3(gm, (O + 7) / 8), 32, 0, st>>>(Z2, B, H, Wb + oW3, theta + ob3, O, 0, Y);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

int nof_mlp_adam(long long P, float* theta, const float* grad, float* m, float* v, int t, float lr, float b1,
                 float b2, float eps, float wd, void* stream) {
    if (P <= 0 || !theta || !grad || !m || !v || t <= 0) {
        nof_set_error("nof_mlp_adam: bad arguments");
        return NOF_EINVAL;
    }
    float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    k_adam32<<<(unsigned)((P + 255) / 256), 256, 0, (cudaStream_t)stream>>>(P, theta, grad, m, v, c1, c2, lr, b1, b2,
                                                                            eps, wd);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

}  // extern "C"
