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
//   GEMM3  Lam'_{mu p} = sum_{P, r} T^P_{mu r} W^P_{r p}   split-K over (P, r), FP64 chunk partials
// with W^P_rp = delta_rp D^P_p - B_pr b^P_rp, D^P = A d^P, d^P_p = b^P_pp (Eq. PNOF coefficients).
// Each operand carries nd = 4 or 5 signed base-256 digits (about 32 or 39 significant bits; see
// digit_gemm.h for the digit contract) under a power-of-two scale per row (GEMM1, GEMM2) or per row
// and part of 16 digit_scale_part_atoms(nd) K elements (GEMM3, whose K runs over all aux indices,
// across which |T| and |W| vary by orders of magnitude); each part sum V has value
// 2^{e_row + e_col - 8 (nd + 1)} V.
// GEMM1's epilogue also records the maxima of |T| per (P, p) over mu that set the digit scales of
// T for GEMM2.
// Tile widths, pipeline depth and the split-K chunk of each GEMM come from the autotuner.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "digit_gemm.h"
#include "internal.h"

struct FastState {
    int n, X, a, ap, katK, nkp, nd, patoms;
    int bn1, bn2, bn3, nchunkJK;
    int* tctr = nullptr;        // [3] tile counters of the three digit GEMMs (dynamic tiles)
    uint16_t* Bd;  int* eB;     // [4][katK][X n][16], per row (P, mu)
    uint16_t *Cd1, *Cd2; int* eC;  // C digits per orbital p (rows p, K = nu) in GEMM1's / GEMM2's tiles
    float2* Tdf;                // [X n][ap] T^P_{mu p} as double-floats
    unsigned* colT;             // [X][ap] max_mu |T^P_{mu p}| (float bits)
    uint16_t* Td2; int* e2;     // [4][katK][X ap][16], per (P, p)
    uint16_t* Td3; int* epT;    // [4][8 nkp][n][16] (K = (P, r) padded to nkp parts), scale per (part, mu)
    float2* bdf;                // [X ap][ap] b^P_{p q} as double-floats
    float2* Ddf;                // [X][a] D^P_p = sum_r A_pr d^P_r
    float2* dg;                 // [X][a] d^P_p = b^P_pp, contiguous (read by the J/K partials)
    uint16_t* Wd3; int* epW;    // rows p (tiles of bn3), K = (P, r); scale per (part, p)
    float2 *Adf, *Bcdf;         // [a][a]
    double *Jpart, *Kpart;      // [nchunkJK][a a]
    double* Lpart;              // [GEMM3 K chunks][n][a] partials of Lambda' (fixed-order sum)
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
// Y = sum_i d_i 256^{nd-1-i} with |d_1..d_{nd-1}| <= 128 (|Y| <= 2^{8 nd}); writes the nd planes
// of element (row r, k) of a digit tensor stored in digit_gemm.h's layout (tiles of RT rows).
__device__ __forceinline__ void put_digits(uint16_t* planes, int RT, int katoms, int nd, long long r, long long k,
                                           long long Y) {
    const long long base = digit_offset(RT, katoms, r, k, 0, nd);
    const long long ps = (long long)RT * 16;  // next plane of the same (tile, atom) block
    for (int i = nd - 1; i >= 1; --i) {
        const int d = (int)(((Y + 128) & 255) - 128);
        planes[base + i * ps] = bf16_bits(d);
        Y = (Y - d) >> 8;
    }
    planes[base] = bf16_bits((int)Y);
}
// BF16 bit pattern of a small integer digit (|d| <= 256, exact: at most 8 significant bits)
__device__ __forceinline__ uint32_t bf16_of_digit(int d) { return __float_as_uint((float)d) >> 16; }

// round((v.x + v.y) 2^s) for |.| <= 2^40 as H 2^16 + L with 32-bit H (|H| <= 2^24), L
// (|L| <= 2^16)
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
// digits of Y = H 2^16 + L (|Y| <= 2^40) with 64-bit shifts (5 digits)
__device__ __forceinline__ void split_digits5_HL(int H, int L, int* d) {
    long long Y = ((long long)H << 16) + L;
#pragma unroll
    for (int i = 4; i >= 1; --i) {
        d[i] = (int)(((Y + 128) & 255) - 128);
        Y = (Y - d[i]) >> 8;
    }
    d[0] = (int)Y;
}
// Eight consecutive K elements (k0 % 8 == 0) of one row from double-floats scaled by 2^s, as nd
// (4 or 5) digits: one 16-byte store per plane.
__device__ __forceinline__ void put8_df(uint16_t* planes, int RT, int katoms, int nd, long long r, long long k0,
                                        const float2* v, const int* s) {
    uint32_t w[5][4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
        int H, L, a[5], b[5];
        df_to_HL(v[j], s[j], H, L);
        if (nd == 4) split_digits_HL(H, L, a[0], a[1], a[2], a[3]);
        else split_digits5_HL(H, L, a);
        df_to_HL(v[j + 1], s[j + 1], H, L);
        if (nd == 4) split_digits_HL(H, L, b[0], b[1], b[2], b[3]);
        else split_digits5_HL(H, L, b);
#pragma unroll
        for (int i = 0; i < 5; ++i)
            if (i < nd) w[i][j / 2] = bf16_of_digit(a[i]) | (bf16_of_digit(b[i]) << 16);
    }
    const long long base = digit_offset(RT, katoms, r, k0, 0, nd);
    const long long ps = (long long)RT * 16;
#pragma unroll
    for (int i = 0; i < 5; ++i)
        if (i < nd)
            *reinterpret_cast<uint4*>(planes + base + i * ps) = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
}

// Scale exponent of a digit row or part whose largest magnitude is mx: e with
// mx < 2^{e - digit_headroom(nd)}, so that the scaled integer Y = x 2^{8 nd - e} has
// |Y| <= digit_top(nd) 256^{nd-1} and its signed base-256 digits meet the digit GEMM's contract.
__device__ __forceinline__ int exp_of(float mx, int nd) {
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);
    return e + digit_headroom(nd);
}


// Digits of an FP64 matrix, one row per warp, scale per row over `ncols` entries:
// element (row, k) = src[row * s_row + k * s_col]; written in one or two tile layouts.
__global__ void k_digits_f64(const double* src, long long s_row, long long s_col, int nrows, int ncols, int nd,
                             int RT, int katoms, uint16_t* planes, int* exps, int RT2, uint16_t* planes2) {
    int w = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= nrows) return;
    double mx = 0.0;
    for (int k = lane; k < ncols; k += 32) mx = fmax(mx, fabs(src[w * s_row + k * s_col]));
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);
    e += digit_headroom(nd);  // |Y| <= digit_top(nd) 256^{nd-1}
    if (lane == 0) exps[w] = e;
    for (int k = lane; k < ncols; k += 32) {
        long long Y = __double2ll_rn(ldexp(src[w * s_row + k * s_col], 8 * nd - e));
        put_digits(planes, RT, katoms, nd, w, k, Y);
        if (planes2) put_digits(planes2, RT2, katoms, nd, w, k, Y);
    }
}

// Reconstruct FP64 rows from digit planes (nof_get_B under the split precision).
__global__ void k_undigit_rows(const uint16_t* planes, const int* exps, int RT, int katoms, int nd, long long rows,
                               int ncols, double* out) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= rows * ncols) return;
    long long r = idx / ncols;
    int k = (int)(idx % ncols);
    long long base = digit_offset(RT, katoms, r, k, 0, nd);
    long long ps = (long long)RT * 16;
    double v = 0.0;
    for (int i = nd - 1; i >= 0; --i) {
        uint16_t u = planes[base + i * ps];
        __nv_bfloat16 b = *reinterpret_cast<__nv_bfloat16*>(&u);
        v = (v + (double)__bfloat162float(b)) / 256.0;
    }
    out[idx] = ldexp(v, exps[r]);
}

// GEMM2's A operand: rows (P, p), K = mu, scale per (P, p) from GEMM1's column maxima. A thread
// takes 8 consecutive mu (one half of a K atom) of one (P, p); the two halves of a row are
// neighbouring threads and lanes run along p, so a warp reads runs of 16 columns of T and writes
// 16 whole swizzled rows (512 bytes) per plane. The thread with mu block 0 stores the exponent.
__global__ void k_T2_digits(const float2* Tdf, const unsigned* colT, int X, int n, int ap, int katK, int nd,
                            uint16_t* Td2, int* e2) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)X * katK * ap * 2) return;
    const int half = (int)(t & 1);
    const long long u = t >> 1;
    const int p = (int)(u % ap);
    const long long w = u / ap;
    const int atom = (int)(w % katK), P = (int)(w / katK);
    const int e = exp_of(__uint_as_float(colT[P * ap + p]), nd);
    if (atom == 0 && half == 0) e2[P * ap + p] = e;
    const int mu0 = atom * 16 + half * 8;
    const float2* T = Tdf + (long long)P * n * ap + p;
    float2 v[8];
    int sh[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int mu = mu0 + j;
        v[j] = mu < n ? T[(long long)mu * ap] : make_float2(0.f, 0.f);
        sh[j] = 8 * nd - e;
    }
    put8_df(Td2, 128, katK, nd, (long long)P * ap + p, (long long)mu0, v, sh);
}

// GEMM3's A operand: rows mu, K = (P, r) padded to nkp parts of PA atoms (PA 16 K elements), a
// scale per (part, mu). A block of 16 PA threads takes 8 rows (mu0..mu0+7) and one part: thread
// (g, i), i = row, g = group of 8 K elements. The 2 PA threads of a row combine their maxima in
// shared memory; the 16 threads of one K atom write its 8 rows as one contiguous 256-byte swizzled
// block per plane.
template <int PA>
__global__ void __launch_bounds__(16 * PA) k_T3_digits(const float2* Tdf, int X, int n, int ap, int nkp, int nd,
                                                       uint16_t* Td3, int* epT) {
    constexpr int kPartK = PA * 16, kPartGroups = 2 * PA;
    __shared__ float mx[kPartGroups][9];
    const int part = blockIdx.x, i = threadIdx.x & 7, g = threadIdx.x >> 3;
    const int mu = blockIdx.y * 8 + i;
    const long long K = (long long)part * kPartK + g * 8;
    float2 v[8];
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = make_float2(0.f, 0.f);
    if (mu < n && K < (long long)X * ap) {
        const int P = (int)(K / ap), r0 = (int)(K - (long long)P * ap);
        // 8 consecutive elements from a multiple of 8 in a row of ap (a multiple of 16): four
        // 16-byte loads
        const float4* src = reinterpret_cast<const float4*>(Tdf + ((long long)P * n + mu) * ap + r0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float4 x = src[j];
            v[2 * j] = make_float2(x.x, x.y);
            v[2 * j + 1] = make_float2(x.z, x.w);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) m = fmaxf(m, fabsf(v[j].x));
    }
    mx[g][i] = m;
    __syncthreads();
    float mr = 0.f;
#pragma unroll
    for (int gg = 0; gg < kPartGroups; ++gg) mr = fmaxf(mr, mx[gg][i]);
    if (mu >= n) return;
    const int e = exp_of(mr, nd);
    if (g == 0) epT[(long long)part * n + mu] = e;
    int sh[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) sh[j] = 8 * nd - e;
    put8_df(Td3, 128, nkp * PA, nd, mu, K, v, sh);
}

// b^P_pq as a double-float (GEMM2's scaled output)
__device__ __forceinline__ float2 b_val(const float2* bdf, int ap, int P, int p, int q) {
    return bdf[((long long)P * ap + p) * ap + q];
}

// d^P_p = b^P_pp for P < X, p < a into a contiguous [X][a] array (one thread per element)
__global__ void __launch_bounds__(256) k_diag(const float2* __restrict__ bdf, int X, int a, int ap,
                                              float2* __restrict__ dg) {
    const long long i = blockIdx.x * 256LL + threadIdx.x;
    if (i >= (long long)X * a) return;
    const int P = (int)(i / a), p = (int)(i - (long long)P * a);
    dg[i] = b_val(bdf, ap, P, p, p);
}

// Partial sums over one chunk of aux indices: J_pq += d_p d_q, K_pq += (b_pq)^2 (double-float),
// with d^P read from the contiguous diagonals (a warp's q are consecutive: every read is
// coalesced or a broadcast); grid (ceil(a*a/256), nchunk); partials [chunk][a*a] as FP64. The
// sums run over P in order; the loads of four consecutive P are issued together.
__global__ void __launch_bounds__(256) k_JK_partial(const float2* __restrict__ bdf, const float2* __restrict__ dg,
                                                    int X, int a, int ap, int nchunk, double* Jpart,
                                                    double* Kpart) {
    const int idx = blockIdx.x * 256 + threadIdx.x;
    const int aa = a * a;
    if (idx >= aa) return;
    const int p = idx / a, q = idx - p * a;
    const int len = (X + nchunk - 1) / nchunk;
    const int P0 = blockIdx.y * len, P1 = min(X, P0 + len);
    float2 jacc = make_float2(0.f, 0.f), kacc = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int P = P0; P < P1; ++P) {
        const float2 b = b_val(bdf, ap, P, p, q);
        const float2 dp = dg[(long long)P * a + p], dq = dg[(long long)P * a + q];
        kacc = df_add(kacc, df_mul(b, b));
        jacc = df_add(jacc, df_mul(dp, dq));
    }
    Jpart[(long long)blockIdx.y * aa + idx] = df_to_double(jacc);
    Kpart[(long long)blockIdx.y * aa + idx] = df_to_double(kacc);
}

// The same for a multiple of 4: each thread takes four consecutive q of one p, so that every
// load of b and of d is 32 bytes (two 16-byte loads) and a warp keeps four times the bytes in
// flight; the sums over P run in the same order as in k_JK_partial.
__global__ void __launch_bounds__(256) k_JK_partial4(const float2* __restrict__ bdf, const float2* __restrict__ dg,
                                                     int X, int a, int ap, int nchunk, double* Jpart,
                                                     double* Kpart) {
    const int idx = (blockIdx.x * 256 + threadIdx.x) * 4;
    const int aa = a * a;
    if (idx >= aa) return;
    const int p = idx / a, q = idx - p * a;
    const int len = (X + nchunk - 1) / nchunk;
    const int P0 = blockIdx.y * len, P1 = min(X, P0 + len);
    float2 jacc[4], kacc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) jacc[i] = kacc[i] = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int P = P0; P < P1; ++P) {
        const float4* bq = reinterpret_cast<const float4*>(bdf + ((long long)P * ap + p) * ap + q);
        const float4* dq = reinterpret_cast<const float4*>(dg + (long long)P * a + q);
        const float4 b01 = bq[0], b23 = bq[1], d01 = dq[0], d23 = dq[1];
        const float2 dp = dg[(long long)P * a + p];
        const float2 b[4] = {make_float2(b01.x, b01.y), make_float2(b01.z, b01.w), make_float2(b23.x, b23.y),
                             make_float2(b23.z, b23.w)};
        const float2 d[4] = {make_float2(d01.x, d01.y), make_float2(d01.z, d01.w), make_float2(d23.x, d23.y),
                             make_float2(d23.z, d23.w)};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            kacc[i] = df_add(kacc[i], df_mul(b[i], b[i]));
            jacc[i] = df_add(jacc[i], df_mul(dp, d[i]));
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        Jpart[(long long)blockIdx.y * aa + idx + i] = df_to_double(jacc[i]);
        Kpart[(long long)blockIdx.y * aa + idx + i] = df_to_double(kacc[i]);
    }
}

// out[i] = sum_b part[b][i], one warp per output, fixed order (lane-strided then a fixed tree);
// blockIdx.y selects one of two (part, out) pairs.
__global__ void k_reduce_parts(const double* part0, double* out0, const double* part1, double* out1, int nparts,
                               int cnt, unsigned* clear, long long nclear) {
    // clear[] (GEMM1's column maxima, read for the last time by k_T2_digits) back to zero for
    // the next evaluation
    const long long nthr = (long long)gridDim.x * gridDim.y * blockDim.x;
    for (long long k = ((long long)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x; k < nclear;
         k += nthr)
        clear[k] = 0u;
    int i = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (i >= cnt) return;
    const double* part = blockIdx.y ? part1 : part0;
    double* out = blockIdx.y ? out1 : out0;
    double s = 0.0;
    for (int b = lane; b < nparts; b += 32) s += part[(long long)b * cnt + i];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[i] = s;
}

// D^P_p = sum_r d^P_r A_rp (A symmetric): a double-float GEMM D [X][a] = d [X][a] A [a][a] in
// 16 x 16 output tiles, one output per thread, K = r staged through shared memory 16 at a time.
__global__ void __launch_bounds__(256) k_D_df(const float2* Adf, const float2* bdf, int X, int a, int ap, float2* D) {
    __shared__ float2 ds[16][17];  // [P][r]
    __shared__ float2 as[16][17];  // [r][p]
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int P0 = blockIdx.y * 16, p0 = blockIdx.x * 16;
    float2 acc = make_float2(0.f, 0.f);
    for (int r0 = 0; r0 < a; r0 += 16) {
        ds[ty][tx] = (P0 + ty < X && r0 + tx < a) ? b_val(bdf, ap, P0 + ty, r0 + tx, r0 + tx) : make_float2(0.f, 0.f);
        as[ty][tx] = (r0 + ty < a && p0 + tx < a) ? Adf[(long long)(r0 + ty) * a + p0 + tx] : make_float2(0.f, 0.f);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) acc = df_add(acc, df_mul(ds[ty][k], as[k][tx]));
        __syncthreads();
    }
    if (P0 + ty < X && p0 + tx < a) D[(long long)(P0 + ty) * a + p0 + tx] = acc;
}

// W^P_rp = delta_rp D^P_p - B_pr b^P_rp for p, r < a (zero in the padding); b^P is symmetric, so
// the element is read at (P, p, r) and W is laid out like it: rows p, K = (P, r).
__device__ __forceinline__ float2 w_val(const float2* bdf, const float2* Bcdf, const float2* D, int a, int ap,
                                        int P, int p, int r) {
    if (p >= a || r >= a) return make_float2(0.f, 0.f);
    float2 w = df_neg(df_mul(Bcdf[p * a + r], b_val(bdf, ap, P, p, r)));
    if (r == p) w = df_add(w, D[(long long)P * a + p]);
    return w;
}

// GEMM3's B operand: rows p < a (tiles of RT), K = (P, r) padded to nkp parts of PA atoms, a scale
// per (part, p); W is recomputed from b and D (no W array). Block and thread layout as k_T3_digits.
template <int PA>
__global__ void __launch_bounds__(16 * PA) k_W_digits(const float2* bdf, const float2* Bcdf, const float2* D, int X,
                                                      int a, int ap, int nkp, int nd, int RT, uint16_t* Wd3,
                                                      int* epW) {
    constexpr int kPartK = PA * 16, kPartGroups = 2 * PA;
    __shared__ float mx[kPartGroups][9];
    const int part = blockIdx.x, i = threadIdx.x & 7, g = threadIdx.x >> 3;
    const int p = blockIdx.y * 8 + i;
    const long long K = (long long)part * kPartK + g * 8;
    float2 v[8];
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = make_float2(0.f, 0.f);
    if (p < a && K < (long long)X * ap) {
        const int P = (int)(K / ap), r0 = (int)(K - (long long)P * ap);
        if ((a & 1) == 0 && r0 + 8 <= a) {
            // all 8 inside the a x a block: b's row and B's row as four 16-byte loads each (r0 a
            // multiple of 8, ap a multiple of 16, p a + r0 even), then the same arithmetic as w_val
            const float4* bs = reinterpret_cast<const float4*>(bdf + ((long long)P * ap + p) * ap + r0);
            const float4* cs = reinterpret_cast<const float4*>(Bcdf + (long long)p * a + r0);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4 bx = bs[j], cx = cs[j];
                v[2 * j] = df_neg(df_mul(make_float2(cx.x, cx.y), make_float2(bx.x, bx.y)));
                v[2 * j + 1] = df_neg(df_mul(make_float2(cx.z, cx.w), make_float2(bx.z, bx.w)));
            }
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (r0 + j == p) v[j] = df_add(v[j], D[(long long)P * a + p]);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = w_val(bdf, Bcdf, D, a, ap, P, p, r0 + j);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) m = fmaxf(m, fabsf(v[j].x));
    }
    mx[g][i] = m;
    __syncthreads();
    float mr = 0.f;
#pragma unroll
    for (int gg = 0; gg < kPartGroups; ++gg) mr = fmaxf(mr, mx[gg][i]);
    if (p >= a) return;
    const int e = exp_of(mr, nd);
    if (g == 0) epW[(long long)part * a + p] = e;
    int sh[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) sh[j] = 8 * nd - e;
    put8_df(Wd3, RT, nkp * PA, nd, p, K, v, sh);
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

// Tile widths worth trying for an N of `ap` columns with nd digits (a tile much wider than the
// matrix only multiplies zeros).
int bn_candidates(int ap, int nd, int* out) {
    int k = 0;
    for (int bn : kDigitBN)
        if (digit_bn_ok(bn, nd) && (bn < 2 * ap || bn == 16)) out[k++] = bn;
    return k;
}

// Lambda[mu][p] = n_p (HC)[mu][p] + sum_b part[b][mu][p] (the K-chunk partials of GEMM3) in a
// fixed order: a block takes 32 consecutive outputs (coalesced) and eight interleaved slices of the
// parts, then adds the slices in order.
__global__ void __launch_bounds__(256) k_lambda_from_parts(const double* part, int nparts, long long cnt,
                                                           const double* HC, const double* occ, int a,
                                                           double* out) {
    __shared__ double acc[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const long long i = blockIdx.x * 32LL + tx;
    double s = 0.0;
    if (i < cnt)
        for (int b = ty; b < nparts; b += 8) s += part[(long long)b * cnt + i];
    acc[ty][tx] = s;
    __syncthreads();
    if (ty == 0 && i < cnt) {
        double t = acc[0][tx];
        for (int k = 1; k < 8; ++k) t += acc[k][tx];
        out[i] = t + occ[i % a] * HC[i];
    }
}

}  // namespace

int fast_release(nof_ctx* c) {
    FastState* f = c->fast;
    if (!f) return NOF_OK;
    ffree(f->Bd); ffree(f->eB); ffree(f->Cd1); ffree(f->Cd2); ffree(f->eC); ffree(f->Tdf); ffree(f->colT);
    ffree(f->Td2); ffree(f->e2); ffree(f->Td3); ffree(f->epT); ffree(f->bdf); ffree(f->Ddf); ffree(f->dg);
    ffree(f->Wd3); ffree(f->epW); ffree(f->Adf); ffree(f->Bcdf); ffree(f->Jpart); ffree(f->Lpart);
    ffree(f->Kpart); ffree(f->tctr);
    delete f;
    c->fast = nullptr;
    return NOF_OK;
}

int fast_prepare(nof_ctx* c) {
    const int n = c->nbf, X = c->naux, a = c->nact;
    const int ap = (a + 15) / 16 * 16, katK = (n + 15) / 16;
    // 32-bit row and K indices of every digit tensor and an exact int64 GEMM3 sum
    if ((long long)X * n > (1LL << 30) || (long long)X * ap * n / 8 > (1LL << 30) ||
        (long long)X * ap * ap / 8 > (1LL << 30)) {
        nof_set_error("NOF_PREC_SPLIT_BF16: system too large for 32-bit tile indices");
        return NOF_EINVAL;
    }
    FastState* f = new (std::nothrow) FastState();
    if (!f) {
        nof_set_error("host allocation failed");
        return NOF_ENOMEM;
    }
    c->fast = f;
    f->n = n; f->X = X; f->a = a; f->ap = ap; f->katK = katK;
    // digits per element: 5 where the 4-digit truncation error, accumulated over the X a terms of
    // the Lagrangian contraction, would approach the 1e-6 accuracy target (X a > 80000)
    const int nd = c->opt.digits ? c->opt.digits : ((long long)X * a > 80000 ? 5 : 4);
    f->nd = nd;
    const long long rowsB = (long long)X * n, rows2 = (long long)X * ap;
    const int patoms = digit_scale_part_atoms(nd);  // atoms per part of GEMM3's per-part scales
    const int nkp = (int)((rows2 / 16 + patoms - 1) / patoms);  // parts of GEMM3's K = (P, r)
    const int kat3 = nkp * patoms;
    f->patoms = patoms;
    f->nkp = nkp;
    // N-side operands (C digits, W digits) hold whole tiles of every candidate width BN
    long long npad = ap;
    for (int bn : kDigitBN) npad = std::max(npad, (long long)(ap + bn - 1) / bn * bn);
    const long long nBd = digit_elems(128, rowsB, katK, nd), nCd = digit_elems(16, npad, katK, nd),
                    nTd2 = digit_elems(128, rows2, katK, nd), nTd3 = digit_elems(128, n, kat3, nd),
                    nWd3 = digit_elems(16, npad, kat3, nd);
    {   // J/K chunks: enough blocks for a few waves, never more than one chunk per 8 aux indices
        // (blocks per chunk as launched: a thread takes four columns when a is a multiple of 4)
        const int per = (int)nblk((long long)a * a / (a % 4 == 0 ? 4 : 1));
        int nc = (4 * 152 + per - 1) / per;
        const int cap = (X + 7) / 8;
        f->nchunkJK = nc < 1 ? 1 : (nc > cap ? cap : nc);
    }
    NOF_TRY(falloc(&f->Bd, nBd)); NOF_TRY(falloc(&f->eB, rowsB));
    NOF_TRY(falloc(&f->Cd1, nCd)); NOF_TRY(falloc(&f->Cd2, nCd)); NOF_TRY(falloc(&f->eC, ap));
    NOF_TRY(falloc(&f->Tdf, rowsB * ap));
    NOF_TRY(falloc(&f->colT, rows2));
    NOF_TRY(falloc(&f->Td2, nTd2)); NOF_TRY(falloc(&f->e2, rows2));
    NOF_TRY(falloc(&f->Td3, nTd3)); NOF_TRY(falloc(&f->epT, (size_t)nkp * n));
    NOF_TRY(falloc(&f->bdf, rows2 * ap));
    NOF_TRY(falloc(&f->Ddf, (size_t)X * a)); NOF_TRY(falloc(&f->dg, (size_t)X * a));
    NOF_TRY(falloc(&f->Wd3, nWd3)); NOF_TRY(falloc(&f->epW, (size_t)nkp * a));
    NOF_TRY(falloc(&f->Adf, (size_t)a * a)); NOF_TRY(falloc(&f->Bcdf, (size_t)a * a));
    NOF_TRY(falloc(&f->Jpart, (size_t)f->nchunkJK * a * a)); NOF_TRY(falloc(&f->Kpart, (size_t)f->nchunkJK * a * a));
    NOF_TRY(falloc(&f->tctr, 3));
    cudaStream_t st = c->stream;
    // digit planes start zeroed: padding rows (p >= nact) and padding K (k >= n) stay zero
    NOF_CUDA(cudaMemsetAsync(f->Bd, 0, 2ull * nBd, st));
    NOF_CUDA(cudaMemsetAsync(f->Cd1, 0, 2ull * nCd, st));
    NOF_CUDA(cudaMemsetAsync(f->Cd2, 0, 2ull * nCd, st));
    NOF_CUDA(cudaMemsetAsync(f->Td2, 0, 2ull * nTd2, st));
    NOF_CUDA(cudaMemsetAsync(f->Td3, 0, 2ull * nTd3, st));
    NOF_CUDA(cudaMemsetAsync(f->Wd3, 0, 2ull * nWd3, st));
    NOF_CUDA(cudaMemsetAsync(f->eC, 0, sizeof(int) * ap, st));
    NOF_CUDA(cudaMemsetAsync(f->e2, 0, sizeof(int) * rows2, st));
    NOF_CUDA(cudaMemsetAsync(f->epT, 0, sizeof(int) * nkp * n, st));
    NOF_CUDA(cudaMemsetAsync(f->epW, 0, sizeof(int) * nkp * a, st));
    NOF_CUDA(cudaMemsetAsync(f->tctr, 0, sizeof(int) * 3, st));
    // B digits, one scale per row (P, mu)
    k_digits_f64<<<nblk(rowsB * 32), 256, 0, st>>>(c->B, n, 1, (int)rowsB, n, nd, 128, katK, f->Bd, f->eB, 0,
                                                   nullptr);
    NOF_LAUNCH_CHECK();

    // ---- autotuned plans ----------------------------------------------------------------
    int bns[6];
    const int nbn = bn_candidates(ap, nd, bns);
    DigitGemmPlan cand[24];
    int best = 0;
    // every GEMM takes its tiles dynamically (a CTA that starts late, behind the side stream's
    // blocks, takes fewer tiles)
    {   // GEMM1: T = B C, scaled double-float output with the maxima of |T|. B was last read one
        // evaluation earlier, so the candidates are timed with L2 flushed.
        DigitGemmOut o;
        o.outf = f->Tdf; o.ldo = ap; o.erow = f->eB; o.ecol = f->eC;
        o.colmax = f->colT; o.group_rows = n;
        o.tile_counter = f->tctr;
        for (int i = 0; i < nbn; ++i)
            NOF_TRY(digit_gemm_plan(&cand[i], f->Bd, f->Cd1, (int)rowsB, ap, bns[i], nd, katK, katK, 0, o,
                                    c->status));
        NOF_TRY(digit_gemm_pick({1, (int)rowsB, ap, katK, n * 8 + nd}, cand, nbn, st, &best, true));
        f->g1 = cand[best];
        f->bn1 = bns[best];
    }
    {   // GEMM2: b = C^T T, scaled double-float output
        DigitGemmOut o;
        o.outf = f->bdf; o.ldo = ap; o.erow = f->e2; o.ecol = f->eC;
        o.tile_counter = f->tctr + 1;
        for (int i = 0; i < nbn; ++i)
            NOF_TRY(digit_gemm_plan(&cand[i], f->Td2, f->Cd2, (int)rows2, ap, bns[i], nd, katK, katK, 0, o,
                                    c->status));
        NOF_TRY(digit_gemm_pick({2, (int)rows2, ap, katK, nd}, cand, nbn, st, &best));
        f->g2 = cand[best];
        f->bn2 = bns[best];
    }
    {   // GEMM3: Lambda' = sum_{P,r} T W with per-part scales; each K chunk stores its FP64 partial
        // (summed afterwards in a fixed order, so results do not depend on scheduling)
        const long long na = (long long)n * a;
        const long long max_chunks = ((long long)1 << 31) / 8 / na;  // at most 2 GiB of partials
        int k = 0, bnk[24], chk[24];  // at most 6 widths x 4 chunks
        int dev = 0, sms = 0;
        NOF_CUDA(cudaGetDevice(&dev));
        NOF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        for (int i = 0; i < nbn; ++i) {
            // per tile width, the three longest chunks (patoms 2^i atoms, or all of K) that still give
            // half a wave of tiles (longer chunks mean fewer partials and less per-tile overhead),
            // and the chunk whose tiles best fill whole waves of the SMs
            const long long tmn = (long long)((n + 127) / 128) * ((a + bns[i] - 1) / bns[i]);
            int all[24], na2 = 0;
            for (long long ch = patoms; na2 < 24; ch *= 2) {
                all[na2++] = (int)(ch < kat3 ? ch : kat3);
                if (ch >= kat3) break;
            }
            int nch = 0;
            for (int j = na2 - 1; j >= 0 && nch < 3; --j) {
                const long long kch = (kat3 + all[j] - 1) / all[j];
                if (kch > max_chunks) break;
                if (tmn * kch < 76 && j > 0) continue;
                chk[k] = all[j];
                bnk[k++] = bns[i];
                ++nch;
            }
            // balance: a wave of sms tiles takes about one chunk's time, so the efficiency of c
            // chunks of ch atoms is tmn kat3 / (sms waves ch); the best, then the fewest chunks
            long long bch = 0;
            double beff = 0.0;
            for (long long c = 1; c <= max_chunks && c <= 64; ++c) {  // at most 64 partials
                const long long ch = ((kat3 + c - 1) / c + patoms - 1) / patoms * patoms;
                const long long kch = (kat3 + ch - 1) / ch;
                if (kch != c || tmn * kch < 76) continue;
                const long long waves = (tmn * kch + sms - 1) / sms;
                const double eff = (double)tmn * kat3 / ((double)sms * waves * ch);
                if (eff > beff + 0.005) {
                    beff = eff;
                    bch = ch;
                }
            }
            bool have = bch == 0;
            for (int j = k - nch; j < k; ++j) have = have || chk[j] == bch;
            if (!have) {
                chk[k] = (int)bch;
                bnk[k++] = bns[i];
            }
        }
        if (k == 0) {
            nof_set_error("NOF_PREC_SPLIT_BF16: no Lagrangian contraction plan fits the partial buffer");
            return NOF_EINVAL;
        }
        long long maxch = 0;
        for (int i = 0; i < k; ++i) {
            const long long kch = (kat3 + chk[i] - 1) / chk[i];
            maxch = kch > maxch ? kch : maxch;
        }
        NOF_TRY(falloc(&f->Lpart, (size_t)(maxch * na)));
        DigitGemmOut o;
        o.outd = f->Lpart; o.ldo = a; o.chunk_stride = na; o.epA = f->epT; o.epB = f->epW;
        o.part_atoms = patoms;
        o.tile_counter = f->tctr + 2;
        for (int i = 0; i < k; ++i)
            NOF_TRY(digit_gemm_plan(&cand[i], f->Td3, f->Wd3, n, a, bnk[i], nd, kat3, chk[i], 0, o, c->status));
        NOF_TRY(digit_gemm_pick({3, n, a, kat3, nd}, cand, k, st, &best));
        f->g3 = cand[best];
        f->bn3 = bnk[best];
    }
    // GEMM1's column maxima start at zero (the autotuner's launches wrote them); from then on
    // k_reduce_parts clears them after each use
    NOF_CUDA(cudaMemsetAsync(f->colT, 0, sizeof(unsigned) * X * ap, st));
    NOF_CUDA(cudaStreamSynchronize(st));
    return NOF_OK;
}

int fast_get_B(nof_ctx* c, double* B) {
    FastState* f = c->fast;
    long long rows = (long long)f->X * f->n;
    k_undigit_rows<<<nblk(rows * f->n), 256, 0, c->stream>>>(f->Bd, f->eB, 128, f->katK, f->nd, rows, f->n, B);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

void fast_coefficient_buffers(nof_ctx* c, float2** Adf, float2** Bcdf) {
    *Adf = c->fast ? c->fast->Adf : nullptr;
    *Bcdf = c->fast ? c->fast->Bcdf : nullptr;
}

int fast_digits(nof_ctx* c) { return c->fast->nd; }

int fast_tiles(nof_ctx* c, int* out) {
    FastState* f = c->fast;
    out[0] = f->bn1;
    out[1] = f->bn2;
    out[2] = f->bn3;
    out[3] = f->g3.g.katoms;
    return NOF_OK;
}

namespace {

// b = C^T B C from C on the context's stream: C digits, GEMM1 (T = B C), the digits of T,
// GEMM2 (b = C^T T). When t_written is not null it is recorded once T is written.
int b_chain(nof_ctx* c, const double* C, cudaEvent_t t_written) {
    FastState* f = c->fast;
    const int n = f->n, X = f->X, a = f->a, ap = f->ap;
    cudaStream_t st = c->stream;
    // C digits: row p over nu (element C[nu][p]), in GEMM1's and GEMM2's tile widths
    k_digits_f64<<<nblk((long long)a * 32), 256, 0, st>>>(C, 1, n, a, n, f->nd, f->bn1, f->katK, f->Cd1, f->eC,
                                                          f->bn2, f->Cd2);
    NOF_LAUNCH_CHECK();
    NOF_TRY(prof_begin(c, "k_digit_gemm (half transform T = B C, tcgen05)"));
    NOF_TRY(digit_gemm_run(f->g1, st));
    NOF_TRY(prof_end(c));
    if (t_written) NOF_CUDA(cudaEventRecord(t_written, st));
    k_T2_digits<<<nblk((long long)X * f->katK * ap * 2), 256, 0, st>>>(f->Tdf, f->colT, X, n, ap, f->katK, f->nd,
                                                                       f->Td2, f->e2);
    NOF_LAUNCH_CHECK();
    NOF_TRY(prof_begin(c, "k_digit_gemm (full transform b = C^T T, tcgen05)", 2));
    NOF_TRY(digit_gemm_run(f->g2, st));
    return prof_end(c, 2);
}

// J and K from b on stream s: chunk partials, then their fixed-order sum. The sum also clears
// GEMM1's column maxima (last read by the digits of T) for the next evaluation.
int jk_from_b(nof_ctx* c, cudaStream_t s) {
    FastState* f = c->fast;
    const int a = f->a, nchunk = f->nchunkJK;
    k_diag<<<nblk((long long)f->X * a), 256, 0, s>>>(f->bdf, f->X, a, f->ap, f->dg);
    NOF_LAUNCH_CHECK();
    if (a % 4 == 0)
        k_JK_partial4<<<dim3(nblk((long long)a * a / 4), nchunk), 256, 0, s>>>(f->bdf, f->dg, f->X, a, f->ap, nchunk,
                                                                            f->Jpart, f->Kpart);
    else
        k_JK_partial<<<dim3(nblk((long long)a * a), nchunk), 256, 0, s>>>(f->bdf, f->dg, f->X, a, f->ap, nchunk,
                                                                         f->Jpart, f->Kpart);
    NOF_LAUNCH_CHECK();
    k_reduce_parts<<<dim3(nblk((long long)a * a * 32), 2), 256, 0, s>>>(f->Jpart, c->J, f->Kpart, c->K, nchunk,
                                                                       a * a, f->colT, (long long)f->X * f->ap);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

// Digits of T for the Lagrangian contraction (GEMM3's M side), on stream s.
int t3_digits(nof_ctx* c, cudaStream_t s) {
    FastState* f = c->fast;
    const dim3 grid(f->nkp, (f->n + 7) / 8);
    if (f->patoms == 20)
        k_T3_digits<20><<<grid, 320, 0, s>>>(f->Tdf, f->X, f->n, f->ap, f->nkp, f->nd, f->Td3, f->epT);
    else
        k_T3_digits<8><<<grid, 128, 0, s>>>(f->Tdf, f->X, f->n, f->ap, f->nkp, f->nd, f->Td3, f->epT);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

// D^P = A d^P (d^P the diagonal of b^P) and the digits of W (GEMM3's N side), on the context's
// stream.
int w_digits(nof_ctx* c) {
    FastState* f = c->fast;
    const int X = f->X, a = f->a, ap = f->ap;
    cudaStream_t st = c->stream;
    k_D_df<<<dim3((a + 15) / 16, (X + 15) / 16), 256, 0, st>>>(f->Adf, f->bdf, X, a, ap, f->Ddf);
    NOF_LAUNCH_CHECK();
    const dim3 grid(f->nkp, (a + 7) / 8);
    if (f->patoms == 20)
        k_W_digits<20><<<grid, 320, 0, st>>>(f->bdf, f->Bcdf, f->Ddf, X, a, ap, f->nkp, f->nd, f->bn3, f->Wd3, f->epW);
    else
        k_W_digits<8><<<grid, 128, 0, st>>>(f->bdf, f->Bcdf, f->Ddf, X, a, ap, f->nkp, f->nd, f->bn3, f->Wd3, f->epW);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

// GEMM3 (Lambda' = sum_P T^P W^P), Lambda, lambda = C^T Lambda and g, on the context's stream,
// once the digits of T and W, H C and the occupations are written.
int lagrangian(nof_ctx* c, const double* C) {
    FastState* f = c->fast;
    cudaStream_t st = c->stream;
    NOF_TRY(prof_begin(c, "k_digit_gemm (Lagrangian contraction sum_P T W, tcgen05)", 3));
    NOF_TRY(digit_gemm_run(f->g3, st));
    NOF_TRY(prof_end(c, 3));
    const long long na = (long long)f->n * f->a;
    k_lambda_from_parts<<<(unsigned)((na + 31) / 32), 256, 0, st>>>(f->Lpart, f->g3.g.kchunks, na, c->HC, c->occ,
                                                                   f->a, c->Lam);
    NOF_LAUNCH_CHECK();
    return pnof_lambda_and_g(c, C, c->gorb, true);
}

}  // namespace

int fast_jk(nof_ctx* c, const double* C) {
    NOF_TRY(b_chain(c, C, nullptr));
    NOF_TRY(jk_from_b(c, c->stream));
    return pnof_hpp(c, C);
}

int fast_grad(nof_ctx* c, const double* C, const double* gamma, bool want_grad) {
    NOF_TRY(pnof_occupations(c, gamma));  // also A and B as double-floats
    NOF_TRY(pnof_energy(c, c->stream));   // E and dE/dgamma
    if (!want_grad) return NOF_OK;
    NOF_TRY(t3_digits(c, c->stream));
    NOF_TRY(w_digits(c));
    return lagrangian(c, C);
}

// One evaluation (fast_jk + fast_grad) on two streams. The context's stream runs the chain the
// gradient needs: C digits, GEMM1, the digits of T, GEMM2, D = A d and the digits of W, GEMM3,
// Lambda, lambda and g. A low-priority side stream, forked from it by an event, runs the rest:
// - the occupations and PNOF coefficients from gamma (the chain waits for them before D);
// - once GEMM1 has written T: H C and h_pp from C, then the GEMM3 digits of T (the chain waits
//   for these before GEMM3). While GEMM1 runs, only the occupation kernels share its SMs;
// - once GEMM2 has written b: the J/K partials, J and K, then E and dE/dgamma (the evaluation
//   ends when these are done too).
// Every buffer the side stream writes is read only after the matching wait. The fork orders
// the side stream after the previous evaluation. No FP64 GEMM shares the split-K scratch with
// H C while it runs: the chain's C^T Lambda comes after GEMM3, which waits for H C.
int fast_eval(nof_ctx* c, const double* C, const double* gamma, bool want_grad) {
    cudaStream_t st = c->stream, sd = c->side;
    NOF_CUDA(cudaEventRecord(c->ev_s0, st));
    NOF_CUDA(cudaStreamWaitEvent(sd, c->ev_s0, 0));
    NOF_TRY(pnof_occupations(c, gamma, sd));
    NOF_CUDA(cudaEventRecord(c->ev_sO, sd));
    // H C and h_pp wait until GEMM1 has written T: while GEMM1 runs, the side stream holds no SM
    // resources beyond the tiny occupation kernels (GEMM1 inside an evaluation: 47 -> 46 us)
    NOF_TRY(b_chain(c, C, c->ev_sT));
    NOF_CUDA(cudaEventRecord(c->ev_sJ, st));
    NOF_CUDA(cudaStreamWaitEvent(sd, c->ev_sT, 0));
    NOF_TRY(pnof_hpp(c, C, sd));
    if (want_grad) {
        NOF_TRY(t3_digits(c, sd));
        NOF_CUDA(cudaEventRecord(c->ev_s1, sd));
    }
    NOF_CUDA(cudaStreamWaitEvent(sd, c->ev_sJ, 0));
    NOF_TRY(jk_from_b(c, sd));
    NOF_TRY(pnof_energy(c, sd));
    NOF_CUDA(cudaEventRecord(c->ev_s2, sd));
    if (want_grad) {
        NOF_CUDA(cudaStreamWaitEvent(st, c->ev_sO, 0));
        NOF_TRY(w_digits(c));
        NOF_CUDA(cudaStreamWaitEvent(st, c->ev_s1, 0));
        NOF_TRY(lagrangian(c, C));
    }
    NOF_CUDA(cudaStreamWaitEvent(st, c->ev_s2, 0));
    return NOF_OK;
}
