// Split-precision evaluation on the tensor cores: the three contractions of the JK step and the
// Lagrangian (orbital transformation of the RI tensor, Single Point Energy section, ERITYP='RI';
// Lagrangian of the Natural Orbital Optimization subsection) run as exact BF16 digit-plane
// GEMMs on tcgen05 (digit_gemm.cu); everything between them is exact integer arithmetic or
// double-float (pairs of FP32) arithmetic, because GB300's FP64 rate (2 FMA/clk/SM) is far
// below what HBM-rate elementwise work needs. FP64 is kept for the small a x a / n x a stages
// (J, K, energy, lambda, the gradients).
//
//   GEMM1  T^P_{mu p}  = sum_nu B^P_{mu nu} C_{nu p}       rows (P, mu), digits of B per row
//   GEMM2  b^P_{p q}   = sum_mu T^P_{mu p} C_{mu q}        rows (P, p), digits of T per (P, p)
//   GEMM3  Lam'_{mu p} = sum_{P, r} T^P_{mu r} W^P_{r p}   split-K over (P, r), integer atomics
// with W^P_rp = delta_rp D^P_p - B_pr b^P_rp, D^P = A d^P, d^P_p = b^P_pp (Eq. PNOF coefficients).
// Each operand carries 4 signed base-256 digits (about 32 significant bits) under a power-of-two
// scale per row; each GEMM result is an exact int64 V with value 2^{e_row + e_col - 40} V.
#include <cuda_bf16.h>

#include <cmath>

#include "digit_gemm.h"
#include "internal.h"

struct FastState {
    int n, X, a, ap, katK, nblk, katoms3;
    uint16_t* Bd;  int* eB;     // [4][katK][X n][16], per row (P, mu)
    uint16_t* Cd;  int* eC;     // [4][katK][ap][16], per orbital p
    long long* Tfix;            // [X n][ap]
    uint16_t* Td2; int* e2;     // [4][katK][X ap][16], per (P, p)
    unsigned* maxT3; int* eT3;  // per mu
    uint16_t* Td3;              // [4][X ap / 16][n][16]
    long long* bfix;            // [X ap][ap]
    float2* Wdf;                // [X][ap][ap]  W^P_rp at (P, p, r)
    unsigned* maxW; int* eW3;   // per p
    uint16_t* Wd3;              // [4][X ap / 16][ap][16]
    long long* Lfix;            // [n][ap]
    float2 *Adf, *Bcdf;         // [a][a]
    double *Jpart, *Kpart;      // [nblk][a a]
    DigitGemmPlan g1, g2, g3;
};

namespace {

inline unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ---- double-float (unevaluated pair of FP32) arithmetic -----------------------------------
__device__ __forceinline__ float2 quick_two_sum(float a, float b) {
    float s = a + b;
    return make_float2(s, b - (s - a));
}
__device__ __forceinline__ float2 two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    return make_float2(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float2 s = two_sum(a.x, b.x);
    return quick_two_sum(s.x, s.y + a.y + b.y);
}
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
    return quick_two_sum(p, e);
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
// 2^e as an FP32 (exact for -126 <= e <= 127; ldexpf handles the rest)
__device__ __forceinline__ float pow2f(int e) {
    if (e >= -126 && e <= 127) return __int_as_float((e + 127) << 23);
    return ldexpf(1.0f, e);
}
// exact integer (|V| < 2^62) times 2^e as a double-float
__device__ __forceinline__ float2 df_from_fix(long long V, int e) {
    float hi = (float)V;
    float lo = (float)(V - (long long)hi);
    if (e >= -126 && e <= 127) {
        float s = pow2f(e);
        return make_float2(hi * s, lo * s);
    }
    return make_float2(ldexpf(hi, e), ldexpf(lo, e));
}
__device__ __forceinline__ double df_to_double(float2 a) { return (double)a.x + (double)a.y; }

// ---- digits ---------------------------------------------------------------------------------
__device__ __forceinline__ uint16_t bf16_bits(int d) {
    __nv_bfloat16 b = __float2bfloat16_rn((float)d);
    return *reinterpret_cast<uint16_t*>(&b);
}
// Y = d0 256^3 + d1 256^2 + d2 256 + d3 with |d1..d3| <= 128; writes the four planes of
// element (row r, k) of an atom-major digit tensor with `rows` rows and `katoms` K atoms.
__device__ __forceinline__ void put_digits(uint16_t* planes, int katoms, long long rows, long long r,
                                           long long k, long long Y) {
    int d3 = (int)(((Y + 128) & 255) - 128);
    Y = (Y - d3) >> 8;
    int d2 = (int)(((Y + 128) & 255) - 128);
    Y = (Y - d2) >> 8;
    int d1 = (int)(((Y + 128) & 255) - 128);
    Y = (Y - d1) >> 8;
    int d0 = (int)Y;
    long long base = ((k >> 4) * rows + r) * 16 + (k & 15);
    long long ps = (long long)katoms * rows * 16;
    planes[base] = bf16_bits(d0);
    planes[base + ps] = bf16_bits(d1);
    planes[base + 2 * ps] = bf16_bits(d2);
    planes[base + 3 * ps] = bf16_bits(d3);
}
// round(V 2^s) for an exact integer V
__device__ __forceinline__ long long shift_round(long long V, int s) {
    if (s >= 0) return V << s;
    int r = -s;
    if (r >= 62) return 0;
    return (V + (1LL << (r - 1))) >> r;
}
__device__ __forceinline__ int exp_of(float mx) {
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);
    return e;  // mx < 2^e
}

// Digits of an FP64 matrix, one row per warp, scale per row over `ncols` entries:
// element (row, k) = src[row * s_row + k * s_col].
__global__ void k_digits_f64(const double* src, long long s_row, long long s_col, int nrows, int ncols,
                             int rows_pad, int katoms, uint16_t* planes, int* exps) {
    int w = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= nrows) return;
    double mx = 0.0;
    for (int k = lane; k < ncols; k += 32) mx = fmax(mx, fabs(src[w * s_row + k * s_col]));
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);
    if (lane == 0) exps[w] = e;
    for (int k = lane; k < ncols; k += 32) {
        long long Y = __double2ll_rn(ldexp(src[w * s_row + k * s_col], 32 - e));
        put_digits(planes, katoms, rows_pad, w, k, Y);
    }
}

// Reconstruct FP64 rows from digit planes (nof_get_B under the split precision).
__global__ void k_undigit_rows(const uint16_t* planes, const int* exps, int katoms, long long rows,
                               int ncols, double* out) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= rows * ncols) return;
    long long r = idx / ncols;
    int k = (int)(idx % ncols);
    long long base = ((long long)(k >> 4) * rows + r) * 16 + (k & 15);
    long long ps = (long long)katoms * rows * 16;
    double v = 0.0;
    for (int i = 3; i >= 0; --i) {
        uint16_t u = planes[base + i * ps];
        __nv_bfloat16 b = *reinterpret_cast<__nv_bfloat16*>(&u);
        v = (v + (double)__bfloat162float(b)) / 256.0;
    }
    out[idx] = ldexp(v, exps[r]);
}

// Block per aux index P: stage T^P (exact fixed point) in shared memory, per-(P,p) scale over mu,
// digits for GEMM2 (rows (P, p), K = mu), and running per-mu maxima for GEMM3's operand.
__global__ void k_T2_digits(const long long* Tfix, const int* eB, const int* eC, int n, int ap,
                            int katK, uint16_t* Td2, int* e2, unsigned* maxT3) {
    extern __shared__ long long Ts[];  // [n][ap + 1] (padded rows)
    __shared__ unsigned colmax[128];
    __shared__ unsigned rowmax[256];
    __shared__ int eBs[256];
    const int P = blockIdx.x;
    const long long base = (long long)P * n * ap;
    for (int i = threadIdx.x; i < ap; i += blockDim.x) colmax[i] = 0u;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        rowmax[i] = 0u;
        eBs[i] = eB[(long long)P * n + i];
    }
    __syncthreads();
    {   // warp w takes rows mu = w, w + nwarps, ...; lane l takes columns p = l, l + 32, ...
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        float cm[4] = {0.f, 0.f, 0.f, 0.f};  // ap <= 128
        float sC[4];
        for (int j = 0; j < 4; ++j) sC[j] = (lane + 32 * j < ap) ? pow2f(eC[lane + 32 * j] - 40) : 0.f;
        for (int mu = warp; mu < n; mu += nw) {
            float rm = 0.f;
            float sB = pow2f(eBs[mu]);
            for (int j = 0; j < 4; ++j) {
                int p = lane + 32 * j;
                if (p >= ap) break;
                long long v = Tfix[base + (long long)mu * ap + p];
                Ts[mu * (ap + 1) + p] = v;
                float f = fabsf((float)v * sC[j] * sB);
                cm[j] = fmaxf(cm[j], f);
                rm = fmaxf(rm, f);
            }
            for (int o = 16; o; o >>= 1) rm = fmaxf(rm, __shfl_xor_sync(0xffffffffu, rm, o));
            if (lane == 0) rowmax[mu] = __float_as_uint(rm);
        }
        for (int j = 0; j < 4; ++j)
            if (lane + 32 * j < ap) atomicMax(&colmax[lane + 32 * j], __float_as_uint(cm[j]));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) atomicMax(&maxT3[i], rowmax[i]);
    for (int p = threadIdx.x; p < ap; p += blockDim.x) e2[(long long)P * ap + p] = exp_of(__uint_as_float(colmax[p]));
    // digits: row (P, p), k = mu; lanes over mu for contiguous 32-byte atom rows
    for (int i = threadIdx.x; i < n * ap; i += blockDim.x) {
        int p = i / n, mu = i - p * n;
        int ep = exp_of(__uint_as_float(colmax[p]));
        long long Y = shift_round(Ts[mu * (ap + 1) + p], eBs[mu] + eC[p] - 8 - ep);
        put_digits(Td2, katK, (long long)gridDim.x * ap, (long long)P * ap + p, mu, Y);
    }
}

// GEMM3's A operand: rows mu, K = (P, r); scale per mu over all (P, r).
__global__ void k_T3_digits(const long long* Tfix, const int* eB, const int* eC, const unsigned* maxT3,
                            int X, int n, int ap, uint16_t* Td3) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long tot = (long long)X * n * ap;
    if (idx >= tot) return;
    long long row = idx / ap;  // P n + mu
    int r = (int)(idx - row * ap);
    long long P = row / n;
    int mu = (int)(row - P * n);
    int e3 = exp_of(__uint_as_float(maxT3[mu]));
    long long Y = shift_round(Tfix[idx], eB[row] + eC[r] - 8 - e3);
    put_digits(Td3, (int)((long long)X * ap / 16), n, mu, P * ap + r, Y);
}

__global__ void k_exps_from_max(const unsigned* mx, int cnt, int* e) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) e[i] = exp_of(__uint_as_float(mx[i]));
}

// b^P_pq as a double-float from GEMM2's fixed-point output
__device__ __forceinline__ float2 b_val(const long long* bfix, const int* e2, const int* eC, int ap, int P,
                                        int p, int q) {
    long long row = (long long)P * ap + p;
    return df_from_fix(bfix[row * ap + q], e2[row] + eC[q] - 40);
}

// Persistent blocks over P: J_pq += d_p d_q, K_pq += (b_pq)^2 in double-float; per-block
// partial sums are written as FP64 and reduced in a fixed order afterwards.
__global__ void __launch_bounds__(256) k_perP_JK(const long long* bfix, const int* e2, const int* eC, int X,
                                                 int a, int ap, double* Jpart, double* Kpart) {
    __shared__ float2 ds[128];
    constexpr int MAXE = 16;  // ap <= 64: ap*ap/256 <= 16 elements per thread
    float2 jacc[MAXE], kacc[MAXE];
    for (int j = 0; j < MAXE; ++j) jacc[j] = kacc[j] = make_float2(0.f, 0.f);
    const int aa = a * a;
    for (int P = blockIdx.x; P < X; P += gridDim.x) {
        __syncthreads();
        for (int p = threadIdx.x; p < a; p += blockDim.x) ds[p] = b_val(bfix, e2, eC, ap, P, p, p);
        __syncthreads();
        for (int j = 0; j < MAXE; ++j) {
            int idx = threadIdx.x + 256 * j;
            if (idx >= aa) break;
            int p = idx / a, q = idx - p * a;
            float2 b = b_val(bfix, e2, eC, ap, P, p, q);
            kacc[j] = df_add(kacc[j], df_mul(b, b));
            jacc[j] = df_add(jacc[j], df_mul(ds[p], ds[q]));
        }
    }
    for (int j = 0; j < MAXE; ++j) {
        int idx = threadIdx.x + 256 * j;
        if (idx >= aa) break;
        Jpart[(long long)blockIdx.x * aa + idx] = df_to_double(jacc[j]);
        Kpart[(long long)blockIdx.x * aa + idx] = df_to_double(kacc[j]);
    }
}

// out[i] = sum_b part[b][i], one warp per output, fixed order (lane-strided then a fixed tree)
__global__ void k_reduce_parts(const double* part, int nparts, int cnt, double* out) {
    int i = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (i >= cnt) return;
    double s = 0.0;
    for (int b = lane; b < nparts; b += 32) s += part[(long long)b * cnt + i];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[i] = s;
}

__global__ void k_to_df(const double* src, int cnt, float2* dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    double v = src[i];
    float hi = (float)v;
    dst[i] = make_float2(hi, (float)(v - (double)hi));
}

// Persistent blocks over P: D^P = A d^P, W^P_rp = delta_rp D^P_p - B_pr b^P_rp (double-float),
// stored at (P, p, r); per-p maxima for the digit scale of GEMM3's B operand.
__global__ void __launch_bounds__(256) k_perP_W(const long long* bfix, const int* e2, const int* eC,
                                                const float2* Adf, const float2* Bcdf, int X, int a, int ap,
                                                float2* Wdf, unsigned* maxW) {
    __shared__ float2 ds[128], Ds[128];
    __shared__ unsigned wmax[128];
    for (int p = threadIdx.x; p < ap; p += blockDim.x) wmax[p] = 0u;
    const int aa = ap * ap;
    for (int P = blockIdx.x; P < X; P += gridDim.x) {
        __syncthreads();
        for (int p = threadIdx.x; p < a; p += blockDim.x) ds[p] = b_val(bfix, e2, eC, ap, P, p, p);
        __syncthreads();
        for (int p = threadIdx.x; p < a; p += blockDim.x) {
            float2 s = make_float2(0.f, 0.f);
            for (int r = 0; r < a; ++r) s = df_add(s, df_mul(Adf[p * a + r], ds[r]));
            Ds[p] = s;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < aa; idx += blockDim.x) {
            int p = idx / ap, r = idx - p * ap;  // stored at (P, p, r)
            float2 w = make_float2(0.f, 0.f);
            if (r < a && p < a) {
                w = df_neg(df_mul(Bcdf[p * a + r], b_val(bfix, e2, eC, ap, P, r, p)));
                if (r == p) w = df_add(w, Ds[p]);
            }
            Wdf[(long long)P * aa + idx] = w;
            unsigned wb = __float_as_uint(fabsf(w.x));
            if ((ap & 31) == 0) {  // the whole warp shares p
                for (int o = 16; o; o >>= 1) wb = max(wb, __shfl_xor_sync(0xffffffffu, wb, o));
                if ((threadIdx.x & 31) == 0) atomicMax(&wmax[p], wb);
            } else {
                atomicMax(&wmax[p], wb);
            }
        }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < ap; p += blockDim.x) atomicMax(&maxW[p], wmax[p]);
}

// GEMM3's B operand: rows p, K = (P, r); scale per p over all (P, r).
__global__ void k_W_digits(const float2* Wdf, const int* eW3, int X, int ap, uint16_t* Wd3) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long tot = (long long)X * ap * ap;
    if (idx >= tot) return;
    long long Pp = idx / ap;  // P ap + p
    int r = (int)(idx - Pp * ap);
    long long P = Pp / ap;
    int p = (int)(Pp - P * ap);
    float2 w = Wdf[idx];
    int s = 32 - eW3[p];
    long long Y = __float2ll_rn(ldexpf(w.x, s)) + __float2ll_rn(ldexpf(w.y, s));
    put_digits(Wd3, (int)((long long)X * ap / 16), ap, p, P * ap + r, Y);
}

__global__ void k_lambda_from_fix(const long long* Lfix, const int* eT3, const int* eW3, int n, int a, int ap,
                                  double* Lam) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n * a) return;
    int mu = (int)(idx / a), p = (int)(idx - (long long)mu * a);
    Lam[idx] = ldexp((double)Lfix[(long long)mu * ap + p], eT3[mu] + eW3[p] - 40);
}

template <class T>
int falloc(T** p, size_t count) {
    cudaError_t e = cudaMalloc((void**)p, (count ? count : 1) * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return nof_cuda_fail(e, "cudaMalloc (split path)", __FILE__, __LINE__);
    }
    return NOF_OK;
}
template <class T>
void ffree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

}  // namespace

int fast_release(nof_ctx* c) {
    FastState* f = c->fast;
    if (!f) return NOF_OK;
    ffree(f->Bd); ffree(f->eB); ffree(f->Cd); ffree(f->eC); ffree(f->Tfix); ffree(f->Td2); ffree(f->e2);
    ffree(f->maxT3); ffree(f->eT3); ffree(f->Td3); ffree(f->bfix); ffree(f->Wdf); ffree(f->maxW);
    ffree(f->eW3); ffree(f->Wd3); ffree(f->Lfix); ffree(f->Adf); ffree(f->Bcdf); ffree(f->Jpart);
    ffree(f->Kpart);
    delete f;
    c->fast = nullptr;
    return NOF_OK;
}

int fast_prepare(nof_ctx* c) {
    const int n = c->nbf, X = c->naux, a = c->nact;
    if (n > 160 || a > 64) {
        nof_set_error("NOF_PREC_SPLIT_BF16 supports nbf <= 160 and nact <= 64 in this build");
        return NOF_EINVAL;
    }
    FastState* f = new (std::nothrow) FastState();
    if (!f) {
        nof_set_error("host allocation failed");
        return NOF_ENOMEM;
    }
    c->fast = f;
    f->n = n; f->X = X; f->a = a;
    f->ap = (a + 15) / 16 * 16;
    f->katK = (n + 15) / 16;
    f->nblk = X < 304 ? X : 304;
    const int ap = f->ap, katK = f->katK;
    const long long rowsB = (long long)X * n, rows2 = (long long)X * ap, kat3 = (long long)X * ap / 16;
    int k3 = 10;
    while (kat3 % k3) --k3;
    f->katoms3 = k3;
    NOF_TRY(falloc(&f->Bd, 4ull * katK * rowsB * 16)); NOF_TRY(falloc(&f->eB, rowsB));
    NOF_TRY(falloc(&f->Cd, 4ull * katK * ap * 16)); NOF_TRY(falloc(&f->eC, ap));
    NOF_TRY(falloc(&f->Tfix, rowsB * ap));
    NOF_TRY(falloc(&f->Td2, 4ull * katK * rows2 * 16)); NOF_TRY(falloc(&f->e2, rows2));
    NOF_TRY(falloc(&f->maxT3, n)); NOF_TRY(falloc(&f->eT3, n));
    NOF_TRY(falloc(&f->Td3, 4ull * kat3 * n * 16));
    NOF_TRY(falloc(&f->bfix, rows2 * ap));
    NOF_TRY(falloc(&f->Wdf, rows2 * ap)); NOF_TRY(falloc(&f->maxW, ap)); NOF_TRY(falloc(&f->eW3, ap));
    NOF_TRY(falloc(&f->Wd3, 4ull * kat3 * ap * 16));
    NOF_TRY(falloc(&f->Lfix, (size_t)n * ap));
    NOF_TRY(falloc(&f->Adf, (size_t)a * a)); NOF_TRY(falloc(&f->Bcdf, (size_t)a * a));
    NOF_TRY(falloc(&f->Jpart, (size_t)f->nblk * a * a)); NOF_TRY(falloc(&f->Kpart, (size_t)f->nblk * a * a));
    cudaStream_t st = c->stream;
    // digit planes start zeroed: padding rows (p >= nact) and padding K (k >= n) stay zero
    NOF_CUDA(cudaMemsetAsync(f->Bd, 0, 8ull * katK * rowsB * 16, st));
    NOF_CUDA(cudaMemsetAsync(f->Cd, 0, 8ull * katK * ap * 16, st));
    NOF_CUDA(cudaMemsetAsync(f->Td2, 0, 8ull * katK * rows2 * 16, st));
    NOF_CUDA(cudaMemsetAsync(f->Td3, 0, 8ull * kat3 * n * 16, st));
    NOF_CUDA(cudaMemsetAsync(f->Wd3, 0, 8ull * kat3 * ap * 16, st));
    NOF_CUDA(cudaMemsetAsync(f->eC, 0, sizeof(int) * ap, st));
    NOF_CUDA(cudaMemsetAsync(f->e2, 0, sizeof(int) * rows2, st));
    // B digits, one scale per row (P, mu)
    k_digits_f64<<<nblk(rowsB * 32), 256, 0, st>>>(c->B, n, 1, (int)rowsB, n, (int)rowsB, katK, f->Bd, f->eB);
    NOF_LAUNCH_CHECK();
    NOF_TRY(digit_gemm_plan(&f->g1, f->Bd, (int)rowsB, f->Cd, ap, katK, katK, (int)rowsB, ap, f->Tfix, ap,
                            false, c->status));
    NOF_TRY(digit_gemm_plan(&f->g2, f->Td2, (int)rows2, f->Cd, ap, katK, katK, (int)rows2, ap, f->bfix, ap,
                            false, c->status));
    NOF_TRY(digit_gemm_plan(&f->g3, f->Td3, n, f->Wd3, ap, (int)kat3, k3, n, ap, f->Lfix, ap, true,
                            c->status));
    NOF_CUDA(cudaFuncSetAttribute(k_T2_digits, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(long long) * 160 * 65)));
    NOF_CUDA(cudaStreamSynchronize(st));
    return NOF_OK;
}

int fast_get_B(nof_ctx* c, double* B) {
    FastState* f = c->fast;
    long long rows = (long long)f->X * f->n;
    k_undigit_rows<<<nblk(rows * f->n), 256, 0, c->stream>>>(f->Bd, f->eB, f->katK, rows, f->n, B);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

int fast_jk(nof_ctx* c, const double* C) {
    FastState* f = c->fast;
    const int n = f->n, X = f->X, a = f->a, ap = f->ap;
    cudaStream_t st = c->stream;
    // C digits: row p over nu (element C[nu][p])
    k_digits_f64<<<nblk((long long)a * 32), 256, 0, st>>>(C, 1, n, a, n, ap, f->katK, f->Cd, f->eC);
    NOF_LAUNCH_CHECK();
    NOF_TRY(prof_begin(c, "k_digit_gemm (half transform T = B C, tcgen05)"));
    NOF_TRY(digit_gemm_run(f->g1, st));
    NOF_TRY(prof_end(c));
    NOF_CUDA(cudaMemsetAsync(f->maxT3, 0, sizeof(unsigned) * n, st));
    k_T2_digits<<<X, 256, sizeof(long long) * n * (ap + 1), st>>>(f->Tfix, f->eB, f->eC, n, ap, f->katK, f->Td2,
                                                            f->e2, f->maxT3);
    NOF_LAUNCH_CHECK();
    NOF_TRY(digit_gemm_run(f->g2, st));
    k_perP_JK<<<f->nblk, 256, 0, st>>>(f->bfix, f->e2, f->eC, X, a, ap, f->Jpart, f->Kpart);
    NOF_LAUNCH_CHECK();
    k_reduce_parts<<<nblk((long long)a * a * 32), 256, 0, st>>>(f->Jpart, f->nblk, a * a, c->J);
    NOF_LAUNCH_CHECK();
    k_reduce_parts<<<nblk((long long)a * a * 32), 256, 0, st>>>(f->Kpart, f->nblk, a * a, c->K);
    NOF_LAUNCH_CHECK();
    return pnof_hpp(c, C);
}

int fast_grad(nof_ctx* c, const double* C, const double* gamma, bool want_grad) {
    FastState* f = c->fast;
    const int n = f->n, X = f->X, a = f->a, ap = f->ap;
    cudaStream_t st = c->stream;
    NOF_TRY(pnof_occupations(c, gamma));
    NOF_TRY(pnof_energy(c));
    if (!want_grad) return NOF_OK;
    k_to_df<<<nblk(a * a), 256, 0, st>>>(c->A, a * a, f->Adf);
    NOF_LAUNCH_CHECK();
    k_to_df<<<nblk(a * a), 256, 0, st>>>(c->Bc, a * a, f->Bcdf);
    NOF_LAUNCH_CHECK();
    NOF_CUDA(cudaMemsetAsync(f->maxW, 0, sizeof(unsigned) * ap, st));
    k_perP_W<<<f->nblk, 256, 0, st>>>(f->bfix, f->e2, f->eC, f->Adf, f->Bcdf, X, a, ap, f->Wdf, f->maxW);
    NOF_LAUNCH_CHECK();
    k_exps_from_max<<<1, 128, 0, st>>>(f->maxW, ap, f->eW3);
    NOF_LAUNCH_CHECK();
    long long nW = (long long)X * ap * ap;
    k_W_digits<<<nblk(nW), 256, 0, st>>>(f->Wdf, f->eW3, X, ap, f->Wd3);
    NOF_LAUNCH_CHECK();
    k_exps_from_max<<<nblk(n, 128), 128, 0, st>>>(f->maxT3, n, f->eT3);
    NOF_LAUNCH_CHECK();
    long long nT = (long long)X * n * ap;
    k_T3_digits<<<nblk(nT), 256, 0, st>>>(f->Tfix, f->eB, f->eC, f->maxT3, X, n, ap, f->Td3);
    NOF_LAUNCH_CHECK();
    NOF_CUDA(cudaMemsetAsync(f->Lfix, 0, sizeof(long long) * n * ap, st));
    NOF_TRY(digit_gemm_run(f->g3, st));
    k_lambda_from_fix<<<nblk((long long)n * a), 256, 0, st>>>(f->Lfix, f->eT3, f->eW3, n, a, ap, c->Lam);
    NOF_LAUNCH_CHECK();
    NOF_TRY(pnof_lambda_and_g(c, C, c->gorb));
    return pnof_gamma_grad(c, c->ggam);
}
