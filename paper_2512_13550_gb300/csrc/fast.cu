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
    float2* Tdf;                // [X n][ap] T^P_{mu p} as double-floats
    uint16_t* Td2; int* e2;     // [4][katK][X ap][16], per (P, p)
    unsigned* maxT3; int* eT3;  // per mu
    uint16_t* Td3;              // [4][X ap / 16][n][16]
    float2* bdf;                // [X ap][ap] b^P_{p q} as double-floats
    float2* Wdf;                // [X][ap][ap]  W^P_rp at (P, p, r)
    unsigned* maxW; int* eW3;   // per p
    uint16_t* Wd3;              // [4][X ap / 16][ap][16]
    long long* Lfix;            // [n][ap]
    float2 *Adf, *Bcdf;         // [a][a]
    double *Jpart, *Kpart;      // [X / 8 chunks][a a]
    float2* ddf;                // [X][a] diagonals d^P_p
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
__device__ __forceinline__ double df_to_double(float2 a) { return (double)a.x + (double)a.y; }

// ---- digits ---------------------------------------------------------------------------------
__device__ __forceinline__ uint16_t bf16_bits(int d) {
    __nv_bfloat16 b = __float2bfloat16_rn((float)d);
    return *reinterpret_cast<uint16_t*>(&b);
}
// Y = d0 256^3 + d1 256^2 + d2 256 + d3 with |d1..d3| <= 128 (|Y| <= 2^32); writes the four
// planes of element (row r, k) of a digit tensor stored in digit_gemm.h's layout (tiles of RT rows).
__device__ __forceinline__ void put_digits(uint16_t* planes, int RT, int katoms, long long r, long long k,
                                           long long Y) {
    int d3 = (int)(((Y + 128) & 255) - 128);
    int Y1 = (int)((Y - d3) >> 8);  // |Y1| <= 2^24 + 1: 32-bit from here on
    int d2 = ((Y1 + 128) & 255) - 128;
    Y1 = (Y1 - d2) >> 8;
    int d1 = ((Y1 + 128) & 255) - 128;
    int d0 = (Y1 - d1) >> 8;
    long long base = digit_offset(RT, katoms, r, k, 0);
    long long ps = (long long)RT * 16;  // next plane of the same (tile, atom) block
    planes[base] = bf16_bits(d0);
    planes[base + ps] = bf16_bits(d1);
    planes[base + 2 * ps] = bf16_bits(d2);
    planes[base + 3 * ps] = bf16_bits(d3);
}
// BF16 bit pattern of a small integer digit (|d| <= 256, exact: at most 8 significant bits)
__device__ __forceinline__ uint32_t bf16_of_digit(int d) { return __float_as_uint((float)d) >> 16; }

// round((v.x + v.y) 2^s) for |.| <= 2^32 as H 2^16 + L with 32-bit H, L (|L| <= 2^15 + 1)
__device__ __forceinline__ void df_to_HL(float2 v, int s, int& H, int& L) {
    const float xs = ldexpf(v.x, s), ys = ldexpf(v.y, s);
    const float h = rintf(xs * (1.0f / 65536.0f));
    H = (int)h;
    L = __float2int_rn(fmaf(-h, 65536.0f, xs) + ys);
}
// digits of Y = H 2^16 + L with 32-bit arithmetic only
__device__ __forceinline__ void split_digits_HL(int H, int L, int& d0, int& d1, int& d2, int& d3) {
    d3 = ((L + 128) & 255) - 128;
    int Y = H * 256 + ((L - d3) >> 8);
    d2 = ((Y + 128) & 255) - 128;
    Y = (Y - d2) >> 8;
    d1 = ((Y + 128) & 255) - 128;
    d0 = (Y - d1) >> 8;
}
// Eight consecutive K elements (k0 % 8 == 0) of one row from double-floats scaled by 2^s.
__device__ __forceinline__ void put8_df(uint16_t* planes, int RT, int katoms, long long r, long long k0,
                                        const float2* v, const int* s) {
    uint32_t w[4][4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
        int H, L, a0, a1, a2, a3, b0, b1, b2, b3;
        df_to_HL(v[j], s[j], H, L);
        split_digits_HL(H, L, a0, a1, a2, a3);
        df_to_HL(v[j + 1], s[j + 1], H, L);
        split_digits_HL(H, L, b0, b1, b2, b3);
        w[0][j / 2] = bf16_of_digit(a0) | (bf16_of_digit(b0) << 16);
        w[1][j / 2] = bf16_of_digit(a1) | (bf16_of_digit(b1) << 16);
        w[2][j / 2] = bf16_of_digit(a2) | (bf16_of_digit(b2) << 16);
        w[3][j / 2] = bf16_of_digit(a3) | (bf16_of_digit(b3) << 16);
    }
    const long long base = digit_offset(RT, katoms, r, k0, 0);
    const long long ps = (long long)RT * 16;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        *reinterpret_cast<uint4*>(planes + base + i * ps) = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
}

__device__ __forceinline__ int exp_of(float mx) {
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);
    return e;  // mx < 2^e
}

// Digits of an FP64 matrix, one row per warp, scale per row over `ncols` entries:
// element (row, k) = src[row * s_row + k * s_col].
__global__ void k_digits_f64(const double* src, long long s_row, long long s_col, int nrows, int ncols,
                             int RT, int katoms, uint16_t* planes, int* exps) {
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
        put_digits(planes, RT, katoms, w, k, Y);
    }
}

// Reconstruct FP64 rows from digit planes (nof_get_B under the split precision).
__global__ void k_undigit_rows(const uint16_t* planes, const int* exps, int RT, int katoms, long long rows,
                               int ncols, double* out) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= rows * ncols) return;
    long long r = idx / ncols;
    int k = (int)(idx % ncols);
    long long base = digit_offset(RT, katoms, r, k, 0);
    long long ps = (long long)RT * 16;
    double v = 0.0;
    for (int i = 3; i >= 0; --i) {
        uint16_t u = planes[base + i * ps];
        __nv_bfloat16 b = *reinterpret_cast<__nv_bfloat16*>(&u);
        v = (v + (double)__bfloat162float(b)) / 256.0;
    }
    out[idx] = ldexp(v, exps[r]);
}

// Block per aux index P (blockDim = (32, 32)): per-(P,p) scale over mu and digits for GEMM2
// (rows (P, p), K = mu), plus running per-mu maxima for GEMM3's operand. T^P is read twice; the
// second read hits L2 (GEMM1 has just written it).
__global__ void __launch_bounds__(1024) k_T2_digits(const float2* Tdf, int n, int ap, int katK, uint16_t* Td2,
                                                    int* e2, unsigned* maxT3) {
    __shared__ float colpart[32][129];  // [ty][p]
    __shared__ int ecol[128];
    const int P = blockIdx.x;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const float2* T = Tdf + (long long)P * n * ap;
    float cm[4] = {0.f, 0.f, 0.f, 0.f};
    for (int mu = ty; mu < n; mu += 32) {  // pass 1: warp ty rows mu, lane tx columns p
        float rm = 0.f;
        for (int j = 0; j < 4; ++j) {
            int p = tx + 32 * j;
            if (p >= ap) break;
            float f = fabsf(T[(long long)mu * ap + p].x);
            cm[j] = fmaxf(cm[j], f);
            rm = fmaxf(rm, f);
        }
        for (int o = 16; o; o >>= 1) rm = fmaxf(rm, __shfl_xor_sync(0xffffffffu, rm, o));
        if (tx == 0) atomicMax(&maxT3[mu], __float_as_uint(rm));
    }
    for (int j = 0; j < 4; ++j)
        if (tx + 32 * j < ap) colpart[ty][tx + 32 * j] = cm[j];
    __syncthreads();
    for (int p = ty * 32 + tx; p < ap; p += 1024) {
        float m = 0.f;
        for (int t = 0; t < 32; ++t) m = fmaxf(m, colpart[t][p]);
        const int e = exp_of(m);
        ecol[p] = e;
        e2[(long long)P * ap + p] = e;
    }
    __syncthreads();
    // pass 2: a thread takes 8 consecutive mu of one p (lanes over p: coalesced loads, one
    // 16-byte store per plane)
    const int nb8 = (n + 7) / 8;
    for (int t = ty * 32 + tx; t < nb8 * ap; t += 1024) {
        const int mb = t / ap, p = t - mb * ap;
        float2 v[8];
        int sh[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int mu = mb * 8 + j;
            v[j] = mu < n ? T[(long long)mu * ap + p] : make_float2(0.f, 0.f);
            sh[j] = 32 - ecol[p];
        }
        put8_df(Td2, 128, katK, (long long)P * ap + p, (long long)mb * 8, v, sh);
    }
}

// GEMM3's A operand: rows mu, K = (P, r); scale per mu over all (P, r). A thread takes 8
// consecutive r of one row (P, mu).
__global__ void k_T3_digits(const float2* Tdf, const unsigned* maxT3, int X, int n, int ap, uint16_t* Td3) {
    const int g8 = ap / 8;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= X * n * g8) return;
    const int row = t / g8, rg = t - row * g8;  // row = P n + mu
    const int P = row / n, mu = row - P * n;
    const int s = 32 - exp_of(__uint_as_float(maxT3[mu]));
    const float2* src = Tdf + (long long)row * ap + rg * 8;
    float2 v[8];
    int sh[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        v[j] = src[j];
        sh[j] = s;
    }
    put8_df(Td3, 128, (int)((long long)X * ap / 16), mu, (long long)P * ap + rg * 8, v, sh);
}

__global__ void k_exps_from_max(const unsigned* mx, int cnt, int* e) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) e[i] = exp_of(__uint_as_float(mx[i]));
}

// b^P_pq as a double-float (GEMM2's scaled output)
__device__ __forceinline__ float2 b_val(const float2* bdf, int ap, int P, int p, int q) {
    return bdf[((long long)P * ap + p) * ap + q];
}

// d^P_p = b^P_pp as double-floats
__global__ void k_diag_df(const float2* bdf, int X, int a, int ap, float2* d) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= X * a) return;
    int P = i / a, p = i - P * a;
    d[i] = b_val(bdf, ap, P, p, p);
}

// Partial sums over a chunk of kJKChunk aux indices: J_pq += d_p d_q, K_pq += (b_pq)^2 (double-
// float); grid (ceil(a*a/256), ceil(X/kJKChunk)); partials [chunk][a*a] as FP64.
constexpr int kJKChunk = 8;
__global__ void __launch_bounds__(256) k_JK_partial(const float2* bdf, const float2* d, int X, int a, int ap,
                                                    double* Jpart, double* Kpart) {
    const int idx = blockIdx.x * 256 + threadIdx.x;
    const int aa = a * a;
    if (idx >= aa) return;
    const int p = idx / a, q = idx - p * a;
    const int P0 = blockIdx.y * kJKChunk, P1 = min(X, P0 + kJKChunk);
    float2 jacc = make_float2(0.f, 0.f), kacc = make_float2(0.f, 0.f);
    for (int P = P0; P < P1; ++P) {
        float2 b = b_val(bdf, ap, P, p, q);
        kacc = df_add(kacc, df_mul(b, b));
        jacc = df_add(jacc, df_mul(d[P * a + p], d[P * a + q]));
    }
    Jpart[(long long)blockIdx.y * aa + idx] = df_to_double(jacc);
    Kpart[(long long)blockIdx.y * aa + idx] = df_to_double(kacc);
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
__global__ void __launch_bounds__(256) k_perP_W(const float2* bdf, const float2* Adf, const float2* Bcdf, int X,
                                                int a, int ap, float2* Wdf, unsigned* maxW) {
    __shared__ float2 ds[128], Ds[128];
    __shared__ unsigned wmax[128];
    for (int p = threadIdx.x; p < ap; p += blockDim.x) wmax[p] = 0u;
    const int aa = ap * ap;
    for (int P = blockIdx.x; P < X; P += gridDim.x) {
        __syncthreads();
        for (int p = threadIdx.x; p < a; p += blockDim.x) ds[p] = b_val(bdf, ap, P, p, p);
        __syncthreads();
        for (int p = threadIdx.x; p < a; p += blockDim.x) {
            float2 s = make_float2(0.f, 0.f);  // D^P_p = sum_r A_pr d_r
            for (int r = 0; r < a; ++r) s = df_add(s, df_mul(Adf[p * a + r], ds[r]));
            Ds[p] = s;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < aa; idx += blockDim.x) {
            int p = idx / ap, r = idx - p * ap;  // stored at (P, p, r)
            float2 w = make_float2(0.f, 0.f);
            if (r < a && p < a) {
                w = df_neg(df_mul(Bcdf[p * a + r], b_val(bdf, ap, P, r, p)));
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

// GEMM3's B operand: rows p, K = (P, r); scale per p over all (P, r). A thread takes 8
// consecutive r of one (P, p).
__global__ void k_W_digits(const float2* Wdf, const int* eW3, int X, int ap, uint16_t* Wd3) {
    const int g8 = ap / 8;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= X * ap * g8) return;
    const int Pp = t / g8, rg = t - Pp * g8;  // Pp = P ap + p
    const int P = Pp / ap, p = Pp - P * ap;
    const int s = 32 - eW3[p];
    const float2* src = Wdf + (long long)Pp * ap + rg * 8;
    float2 v[8];
    int sh[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        v[j] = src[j];
        sh[j] = s;
    }
    put8_df(Wd3, ap, (int)((long long)X * ap / 16), p, (long long)P * ap + rg * 8, v, sh);
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
    ffree(f->Bd); ffree(f->eB); ffree(f->Cd); ffree(f->eC); ffree(f->Tdf); ffree(f->Td2); ffree(f->e2);
    ffree(f->maxT3); ffree(f->eT3); ffree(f->Td3); ffree(f->bdf); ffree(f->Wdf); ffree(f->maxW);
    ffree(f->eW3); ffree(f->Wd3); ffree(f->Lfix); ffree(f->Adf); ffree(f->Bcdf); ffree(f->Jpart);
    ffree(f->Kpart); ffree(f->ddf);
    delete f;
    c->fast = nullptr;
    return NOF_OK;
}

int fast_prepare(nof_ctx* c) {
    const int n = c->nbf, X = c->naux, a = c->nact;
    if (n > 320 || a > 64) {
        nof_set_error("NOF_PREC_SPLIT_BF16 supports nbf <= 320 and nact <= 64 in this build");
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
    const long long nBd = digit_elems(128, rowsB, katK), nCd = digit_elems(ap, ap, katK),
                    nTd2 = digit_elems(128, rows2, katK), nTd3 = digit_elems(128, n, (int)kat3),
                    nWd3 = digit_elems(ap, ap, (int)kat3);
    NOF_TRY(falloc(&f->Bd, nBd)); NOF_TRY(falloc(&f->eB, rowsB));
    NOF_TRY(falloc(&f->Cd, nCd)); NOF_TRY(falloc(&f->eC, ap));
    NOF_TRY(falloc(&f->Tdf, rowsB * ap));
    NOF_TRY(falloc(&f->Td2, nTd2)); NOF_TRY(falloc(&f->e2, rows2));
    NOF_TRY(falloc(&f->maxT3, n)); NOF_TRY(falloc(&f->eT3, n));
    NOF_TRY(falloc(&f->Td3, nTd3));
    NOF_TRY(falloc(&f->bdf, rows2 * ap));
    NOF_TRY(falloc(&f->Wdf, rows2 * ap)); NOF_TRY(falloc(&f->maxW, ap)); NOF_TRY(falloc(&f->eW3, ap));
    NOF_TRY(falloc(&f->Wd3, nWd3));
    NOF_TRY(falloc(&f->Lfix, (size_t)n * ap));
    NOF_TRY(falloc(&f->Adf, (size_t)a * a)); NOF_TRY(falloc(&f->Bcdf, (size_t)a * a));
    const size_t nchunk = (size_t)(X + 7) / 8;
    NOF_TRY(falloc(&f->Jpart, nchunk * a * a)); NOF_TRY(falloc(&f->Kpart, nchunk * a * a));
    NOF_TRY(falloc(&f->ddf, (size_t)X * a));
    cudaStream_t st = c->stream;
    // digit planes start zeroed: padding rows (p >= nact) and padding K (k >= n) stay zero
    NOF_CUDA(cudaMemsetAsync(f->Bd, 0, 2ull * nBd, st));
    NOF_CUDA(cudaMemsetAsync(f->Cd, 0, 2ull * nCd, st));
    NOF_CUDA(cudaMemsetAsync(f->Td2, 0, 2ull * nTd2, st));
    NOF_CUDA(cudaMemsetAsync(f->Td3, 0, 2ull * nTd3, st));
    NOF_CUDA(cudaMemsetAsync(f->Wd3, 0, 2ull * nWd3, st));
    NOF_CUDA(cudaMemsetAsync(f->eC, 0, sizeof(int) * ap, st));
    NOF_CUDA(cudaMemsetAsync(f->e2, 0, sizeof(int) * rows2, st));
    // B digits, one scale per row (P, mu)
    k_digits_f64<<<nblk(rowsB * 32), 256, 0, st>>>(c->B, n, 1, (int)rowsB, n, 128, katK, f->Bd, f->eB);
    NOF_LAUNCH_CHECK();
    NOF_TRY(digit_gemm_plan_scaled(&f->g1, f->Bd, f->Cd, ap, katK, (int)rowsB, ap, f->Tdf, ap, f->eB, f->eC,
                                   c->status));
    NOF_TRY(digit_gemm_plan_scaled(&f->g2, f->Td2, f->Cd, ap, katK, (int)rows2, ap, f->bdf, ap, f->e2, f->eC,
                                   c->status));
    NOF_TRY(digit_gemm_plan(&f->g3, f->Td3, f->Wd3, ap, (int)kat3, k3, n, ap, f->Lfix, ap, true, c->status));
    NOF_CUDA(cudaStreamSynchronize(st));
    return NOF_OK;
}

int fast_get_B(nof_ctx* c, double* B) {
    FastState* f = c->fast;
    long long rows = (long long)f->X * f->n;
    k_undigit_rows<<<nblk(rows * f->n), 256, 0, c->stream>>>(f->Bd, f->eB, 128, f->katK, rows, f->n, B);
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
    k_T2_digits<<<X, dim3(32, 32), 0, st>>>(f->Tdf, n, ap, f->katK, f->Td2, f->e2, f->maxT3);
    NOF_LAUNCH_CHECK();
    NOF_TRY(digit_gemm_run(f->g2, st));
    k_diag_df<<<nblk((long long)X * a), 256, 0, st>>>(f->bdf, X, a, ap, f->ddf);
    NOF_LAUNCH_CHECK();
    const int nchunk = (X + kJKChunk - 1) / kJKChunk;
    k_JK_partial<<<dim3(nblk((long long)a * a), nchunk), 256, 0, st>>>(f->bdf, f->ddf, X, a, ap, f->Jpart,
                                                                      f->Kpart);
    NOF_LAUNCH_CHECK();
    k_reduce_parts<<<nblk((long long)a * a * 32), 256, 0, st>>>(f->Jpart, nchunk, a * a, c->J);
    NOF_LAUNCH_CHECK();
    k_reduce_parts<<<nblk((long long)a * a * 32), 256, 0, st>>>(f->Kpart, nchunk, a * a, c->K);
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
    k_perP_W<<<X, 256, 0, st>>>(f->bdf, f->Adf, f->Bcdf, X, a, ap, f->Wdf, f->maxW);
    NOF_LAUNCH_CHECK();
    k_exps_from_max<<<1, 128, 0, st>>>(f->maxW, ap, f->eW3);
    NOF_LAUNCH_CHECK();
    k_W_digits<<<nblk((long long)X * ap * (ap / 8)), 256, 0, st>>>(f->Wdf, f->eW3, X, ap, f->Wd3);
    NOF_LAUNCH_CHECK();
    k_exps_from_max<<<nblk(n, 128), 128, 0, st>>>(f->maxT3, n, f->eT3);
    NOF_LAUNCH_CHECK();
    k_T3_digits<<<nblk((long long)X * n * (ap / 8)), 256, 0, st>>>(f->Tdf, f->maxT3, X, n, ap, f->Td3);
    NOF_LAUNCH_CHECK();
    NOF_CUDA(cudaMemsetAsync(f->Lfix, 0, sizeof(long long) * n * ap, st));
    NOF_TRY(digit_gemm_run(f->g3, st));
    k_lambda_from_fix<<<nblk((long long)n * a), 256, 0, st>>>(f->Lfix, f->eT3, f->eW3, n, a, ap, c->Lam);
    NOF_LAUNCH_CHECK();
    NOF_TRY(pnof_lambda_and_g(c, C, c->gorb));
    return pnof_gamma_grad(c, c->ggam);
}
