// FP64 dense building blocks: strided GEMM (plain and split-K), Cholesky factor of the aux
// metric and its inverse, Newton-Schulz inverse square root, exponential of an antisymmetric
// matrix by scaling and squaring. All FP64 SIMT; these are the plain path and the set-up.
#include <cmath>
#include <vector>

#include "internal.h"

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

__device__ __forceinline__ long long a_off(const Gemm64& g, int m, int k) {
    int k1 = k / g.K0, k0 = k - k1 * g.K0;
    return (long long)m * g.sAm + (long long)k0 * g.sAk0 + (long long)k1 * g.sAk1;
}
__device__ __forceinline__ long long b_off(const Gemm64& g, int n, int k) {
    int k1 = k / g.K0, k0 = k - k1 * g.K0;
    return (long long)n * g.sBn + (long long)k0 * g.sBk0 + (long long)k1 * g.sBk1;
}

// 64x64 output tile per CTA, 256 threads, 4x4 outputs per thread (rows ty+16i, cols tx+16j).
// If `work` is non-null the CTA writes its raw partial sum for K range [k_lo, k_hi) into
// work[split][M][N]; otherwise it applies alpha/beta into C.
__global__ void __launch_bounds__(256) k_gemm64(Gemm64 g, int splits, double* work) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int z = blockIdx.z;
    const int bidx = z / splits, split = z - bidx * splits;
    const double* A = g.A + (long long)bidx * g.bA;
    const double* Bm = g.B + (long long)bidx * g.bB;
    int kchunk = (g.K + splits - 1) / splits;
    kchunk = (kchunk + BK - 1) / BK * BK;
    const int k_lo = split * kchunk;
    int k_hi = min(g.K, k_lo + kchunk);
    if (g.a_lower) k_hi = min(k_hi, m0 + BM);  // lower-triangular A: nothing past the diagonal block
    const bool a_kfast = (g.sAk0 == 1);
    const bool b_nfast = (g.sBn == 1);
    double acc[4][4] = {};
    for (int kt = k_lo; kt < k_hi; kt += BK) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            int e = tid + 256 * l;
            int mm, kk;
            if (a_kfast) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
            int m = m0 + mm, k = kt + kk;
            As[kk][mm] = (m < g.M && k < k_hi) ? A[a_off(g, m, k)] : 0.0;
            int nn, kb;
            if (b_nfast) { nn = e % BN; kb = e / BN; } else { kb = e % BK; nn = e / BK; }
            int n = n0 + nn, kq = kt + kb;
            Bs[kb][nn] = (n < g.N && kq < k_hi) ? Bm[b_off(g, n, kq)] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
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
            if (work) {
                work[((long long)split * g.M + m) * g.N + n] = acc[i][j];
            } else {
                double* Cp = g.C + (long long)bidx * g.bC + (long long)m * g.sCm + (long long)n * g.sCn;
                double v = g.alpha * acc[i][j];
                if (g.beta != 0.0) v += g.beta * *Cp;
                *Cp = v;
            }
        }
    }
}

// Skinny outputs: 16x16 tile per CTA, one output per thread, K range split over grid z.
// Writes raw partials to work[split][M][N].
__global__ void __launch_bounds__(256) k_gemm64_small(Gemm64 g, int splits, double* work) {
    __shared__ double As[16][17];
    __shared__ double Bs[16][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * 16, n0 = blockIdx.x * 16, split = blockIdx.z;
    int kchunk = (g.K + splits - 1) / splits;
    kchunk = (kchunk + 15) / 16 * 16;
    const int k_lo = split * kchunk, k_hi = min(g.K, k_lo + kchunk);
    const bool a_kfast = (g.sAk0 == 1);
    double acc = 0.0;
    for (int kt = k_lo; kt < k_hi; kt += 16) {
        {   // A tile: rows m0.., k kt..
            int mm = a_kfast ? ty : tx, kk = a_kfast ? tx : ty;
            int m = m0 + mm, k = kt + kk;
            As[kk][mm] = (m < g.M && k < k_hi) ? g.A[a_off(g, m, k)] : 0.0;
            int nn = (g.sBn == 1) ? tx : ty, kb = (g.sBn == 1) ? ty : tx;
            int n = n0 + nn, kq = kt + kb;
            Bs[kb][nn] = (n < g.N && kq < k_hi) ? g.B[b_off(g, n, kq)] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) acc = fma(As[kk][ty], Bs[kk][tx], acc);
        __syncthreads();
    }
    int m = m0 + ty, n = n0 + tx;
    if (m < g.M && n < g.N) work[((long long)split * g.M + m) * g.N + n] = acc;
}

__global__ void k_splitk_reduce(Gemm64 g, int splits, const double* work) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long MN = (long long)g.M * g.N;
    if (i >= MN) return;
    int m = (int)(i / g.N), n = (int)(i - (long long)m * g.N);
    double s = 0.0;
    for (int p = 0; p < splits; ++p) s += work[p * MN + i];
    double* Cp = g.C + (long long)m * g.sCm + (long long)n * g.sCn;
    double v = g.alpha * s;
    if (g.beta != 0.0) v += g.beta * *Cp;
    *Cp = v;
}

// ---- Cholesky (left-looking, one launch per column) ------------------------------------
// Row i >= j of column j: L_ij = (V_ij - sum_{k<j} L_ik L_jk) / L_jj. One warp per row;
// every CTA recomputes the pivot of column j so no grid-wide barrier is needed.
__global__ void k_chol_col(double* L, double* pivots, int X, int j, double thresh, int* status) {
    __shared__ double piv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (warp == 0) {
        double s = 0.0;
        for (int k = lane; k < j; k += 32) s = fma(L[(long long)j * X + k], L[(long long)j * X + k], s);
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            double d = L[(long long)j * X + j] - s;
            if (!(d > thresh)) {
                if (blockIdx.x == 0) atomicOr(status, NOF_DEV_ILLCOND);
                d = thresh > 0 ? thresh : 1e-300;
            }
            piv = sqrt(d);
        }
    }
    __syncthreads();
    for (int i = j + 1 + blockIdx.x * nw + warp; i < X; i += gridDim.x * nw) {
        double s = 0.0;
        for (int k = lane; k < j; k += 32) s = fma(L[(long long)i * X + k], L[(long long)j * X + k], s);
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) L[(long long)i * X + j] = (L[(long long)i * X + j] - s) / piv;
    }
    // the diagonal itself is written after the last column (other CTAs still read V_jj)
    if (blockIdx.x == 0 && threadIdx.x == 0) pivots[j] = piv;
}

__global__ void k_set_diag(double* L, const double* pivots, int X) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < X) L[(long long)j * X + j] = pivots[j];
}

// Forward substitution L Z = I, one thread per column j of Z = L^{-1} (lower triangular).
__global__ void k_tri_inverse(const double* L, double* Z, int X) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= X) return;
    for (int i = 0; i < j; ++i) Z[(long long)i * X + j] = 0.0;
    for (int i = j; i < X; ++i) {
        double s = (i == j) ? 1.0 : 0.0;
        for (int k = j; k < i; ++k) s = fma(-L[(long long)i * X + k], Z[(long long)k * X + j], s);
        Z[(long long)i * X + j] = s / L[(long long)i * X + i];
    }
}

__global__ void k_max_diag(const double* V, int X, double* out) {
    __shared__ double red[256];
    double m = 0.0;
    for (int i = threadIdx.x; i < X; i += blockDim.x) m = fmax(m, V[(long long)i * X + i]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// ---- elementwise helpers ----------------------------------------------------------------
__global__ void k_frob(const double* A, long long n, double* out) {
    __shared__ double red[256];
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) s = fma(A[i], A[i], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sqrt(red[0]);
}

// T = 1.5 I - 0.5 P
__global__ void k_ns_mid(const double* P, double* T, int n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)n * n) return;
    int r = (int)(i / n), c = (int)(i % n);
    T[i] = ((r == c) ? 1.5 : 0.0) - 0.5 * P[i];
}
// U = I + A / k  (A already holds z U)
__global__ void k_axpy_identity(const double* A, double inv_k, double* U, int n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)n * n) return;
    int r = (int)(i / n), c = (int)(i % n);
    U[i] = ((r == c) ? 1.0 : 0.0) + A[i] * inv_k;
}
__global__ void k_scale(const double* A, double s, double* out, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = A[i] * s;
}

inline unsigned blocks_for(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

Gemm64 square_gemm(const double* A, const double* B, double* C, int n, double* work = nullptr,
                   size_t work_cap = 0) {
    Gemm64 g;
    g.M = n; g.N = n; g.K = n;
    g.A = A; g.sAm = n; g.sAk0 = 1;
    g.B = B; g.sBn = 1; g.sBk0 = n;
    g.C = C; g.sCm = n; g.sCn = 1;
    g.work = work;
    g.work_cap = work_cap;
    return g;
}

// ---- symmetric eigendecomposition: cyclic Jacobi, round-robin pair order ---------------------
// One CTA. A (n x n, symmetric, destroyed) and V (n x n, starts as I) live in global memory. In
// each round the n/2 disjoint pairs (p, q) of a round-robin tournament (position 0 fixed, the
// others rotating) each get a Givens rotation zeroing A_pq (Golub & Van Loan, Matrix
// Computations, Sec. 8.5: t = sign(th)/(|th| + sqrt(th^2 + 1)), th = (A_qq - A_pp)/(2 A_pq));
// the rotations are applied to rows, then columns, of A and to the columns of V. Sweeps stop
// when the off-diagonal Frobenius norm falls below tol times the total norm, or after max_sweeps.
__global__ void __launch_bounds__(1024) k_jacobi(double* A, double* V, int n, int max_sweeps, double tol,
                                                 int* sweeps_out) {
    extern __shared__ double sh[];
    const int m = n + (n & 1);      // players (a dummy index n when n is odd)
    double* cs = sh;                // [m/2] cos
    double* sn = sh + m / 2;        // [m/2] sin
    int* pp = (int*)(sn + m / 2);   // [m/2]
    int* qq = pp + m / 2;           // [m/2]
    __shared__ double red[1024];
    __shared__ int done;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (long long i = tid; i < (long long)n * n; i += nt) V[i] = ((i / n) == (i % n)) ? 1.0 : 0.0;
    if (tid == 0) done = 0;
    __syncthreads();
    int sweep = 0;
    for (; sweep < max_sweeps && !done; ++sweep) {
        for (int r = 0; r < m - 1; ++r) {
            // pairs of round r: position 0 holds player 0, positions 1..m-1 hold players rotated by r
            for (int i = tid; i < m / 2; i += nt) {
                int a = (i == 0) ? 0 : 1 + (i - 1 + r) % (m - 1);
                int b = 1 + (m - 2 - i + r) % (m - 1);
                int p = min(a, b), q = max(a, b);
                double c = 1.0, s = 0.0;
                if (q < n) {
                    double apq = A[(long long)p * n + q];
                    if (fabs(apq) > 1e-300) {
                        double th = (A[(long long)q * n + q] - A[(long long)p * n + p]) / (2.0 * apq);
                        double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        s = t * c;
                    }
                }
                cs[i] = c; sn[i] = s; pp[i] = p; qq[i] = q;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (long long e = tid; e < (long long)(m / 2) * n; e += nt) {
                int i = (int)(e / n), k = (int)(e % n);
                int p = pp[i], q = qq[i];
                if (q >= n) continue;
                double c = cs[i], s = sn[i];
                double ap = A[(long long)p * n + k], aq = A[(long long)q * n + k];
                A[(long long)p * n + k] = c * ap - s * aq;
                A[(long long)q * n + k] = s * ap + c * aq;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (long long e = tid; e < (long long)(m / 2) * n; e += nt) {
                int i = (int)(e / n), k = (int)(e % n);
                int p = pp[i], q = qq[i];
                if (q >= n) continue;
                double c = cs[i], s = sn[i];
                double ap = A[(long long)k * n + p], aq = A[(long long)k * n + q];
                A[(long long)k * n + p] = c * ap - s * aq;
                A[(long long)k * n + q] = s * ap + c * aq;
                double vp = V[(long long)k * n + p], vq = V[(long long)k * n + q];
                V[(long long)k * n + p] = c * vp - s * vq;
                V[(long long)k * n + q] = s * vp + c * vq;
            }
            __syncthreads();
        }
        // convergence: off-diagonal vs total Frobenius norm
        double off = 0.0, tot = 0.0;
        for (long long i = tid; i < (long long)n * n; i += nt) {
            double v = A[i] * A[i];
            tot += v;
            if ((i / n) != (i % n)) off += v;
        }
        red[tid] = off;
        __syncthreads();
        for (int o = nt / 2; o; o >>= 1) {
            if (tid < o) red[tid] += red[tid + o];
            __syncthreads();
        }
        double offs = red[0];
        __syncthreads();
        red[tid] = tot;
        __syncthreads();
        for (int o = nt / 2; o; o >>= 1) {
            if (tid < o) red[tid] += red[tid + o];
            __syncthreads();
        }
        if (tid == 0 && offs <= tol * tol * red[0]) done = 1;
        __syncthreads();
    }
    if (tid == 0) *sweeps_out = sweep;
}

// Ascending order of the eigenvalues diag(A) (ties keep index order) and the matching columns:
// out[mu][j] = V[mu][perm[j]], w[j] = A[perm[j]][perm[j]].
__global__ void k_eig_sort(const double* A, const double* V, int n, double* out, double* w) {
    extern __shared__ int perm[];
    if (threadIdx.x == 0) {
        for (int i = 0; i < n; ++i) perm[i] = i;
        for (int i = 1; i < n; ++i) {  // insertion sort (stable)
            int x = perm[i];
            double ax = A[(long long)x * n + x];
            int j = i - 1;
            while (j >= 0 && A[(long long)perm[j] * n + perm[j]] > ax) {
                perm[j + 1] = perm[j];
                --j;
            }
            perm[j + 1] = x;
        }
    }
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
        int mu = (int)(e / n), j = (int)(e % n);
        out[e] = V[(long long)mu * n + perm[j]];
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) w[j] = A[(long long)perm[j] * n + perm[j]];
}

}  // namespace

// Eigendecomposition of the symmetric A (destroyed): vectors (ascending eigenvalues) into Vout
// (columns), eigenvalues into w. Work: Vwork (n x n).
int sym_eig(double* A, double* Vwork, double* Vout, double* w, int n, int* sweeps_dev, cudaStream_t st) {
    const int m = n + (n & 1);
    size_t shm = (size_t)(m / 2) * (2 * sizeof(double) + 2 * sizeof(int));
    if (shm > 48 * 1024) NOF_CUDA(cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    k_jacobi<<<1, 1024, shm, st>>>(A, Vwork, n, 30, 1e-14, sweeps_dev);
    NOF_LAUNCH_CHECK();
    k_eig_sort<<<1, 1024, (size_t)n * sizeof(int), st>>>(A, Vwork, n, Vout, w);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

int gemm64_small_splits(const Gemm64& g) {
    if (g.M <= 0 || g.N <= 0 || g.batch != 1 || !g.work) return 0;
    const long long tiles = (long long)((g.N + BN - 1) / BN) * ((g.M + BM - 1) / BM);
    if (tiles >= 304) return 0;
    // small output: 16x16 tiles and a K split so that about 600 CTAs share the work
    const long long t16 = (long long)((g.N + 15) / 16) * ((g.M + 15) / 16);
    long long splits = (608 + t16 - 1) / t16;
    const long long maxs = (g.K + 15) / 16;
    if (splits > maxs) splits = maxs;
    const long long cap = (long long)(g.work_cap / ((size_t)g.M * g.N));
    if (splits > cap) splits = cap;
    return splits >= 1 ? (int)splits : 0;
}

int gemm64_small_partials(const Gemm64& g, int splits, cudaStream_t st) {
    dim3 grid((g.N + 15) / 16, (g.M + 15) / 16, (unsigned)splits);
    k_gemm64_small<<<grid, 256, 0, st>>>(g, splits, g.work);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

int gemm64(const Gemm64& g, cudaStream_t st) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return NOF_OK;
    if (const int splits = gemm64_small_splits(g)) {
        NOF_TRY(gemm64_small_partials(g, splits, st));
        k_splitk_reduce<<<blocks_for((long long)g.M * g.N), 256, 0, st>>>(g, splits, g.work);
        NOF_LAUNCH_CHECK();
        return NOF_OK;
    }
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.batch);
    if (grid.y > 65535u || grid.z > 65535u) {
        nof_set_error("gemm64: grid too large");
        return NOF_EINVAL;
    }
    k_gemm64<<<grid, 256, 0, st>>>(g, 1, nullptr);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

int gemm64_splitk(const Gemm64& g, int splits, double* work, cudaStream_t st) {
    if (g.batch != 1) {
        nof_set_error("gemm64_splitk: batch must be 1");
        return NOF_EINVAL;
    }
    if (splits <= 1) return gemm64(g, st);
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, splits);
    k_gemm64<<<grid, 256, 0, st>>>(g, splits, work);
    NOF_LAUNCH_CHECK();
    k_splitk_reduce<<<blocks_for((long long)g.M * g.N), 256, 0, st>>>(g, splits, work);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

// V (X x X, overwritten by L in its lower triangle) -> Linv. Pivots below 1e-14 of the
// largest diagonal element mark the metric as numerically singular.
int cholesky_inverse(double* V, double* Linv, int X, int* status, cudaStream_t st) {
    double* dmax = Linv;  // scratch: first element, overwritten later
    k_max_diag<<<1, 256, 0, st>>>(V, X, dmax);
    NOF_LAUNCH_CHECK();
    double h_max = 0.0;
    NOF_CUDA(cudaMemcpyAsync(&h_max, dmax, sizeof(double), cudaMemcpyDeviceToHost, st));
    NOF_CUDA(cudaStreamSynchronize(st));
    const double thresh = 1e-14 * h_max;
    for (int j = 0; j < X; ++j) {
        int rows = X - j - 1;
        int blocks = rows <= 0 ? 1 : (rows + 7) / 8;
        if (blocks > 1024) blocks = 1024;
        k_chol_col<<<blocks, 256, 0, st>>>(V, Linv, X, j, thresh, status);
        NOF_LAUNCH_CHECK();
    }
    k_set_diag<<<blocks_for(X, 128), 128, 0, st>>>(V, Linv, X);  // pivots sat in Linv[0..X)
    NOF_LAUNCH_CHECK();
    k_tri_inverse<<<blocks_for(X, 128), 128, 0, st>>>(V, Linv, X);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

// Coupled Newton-Schulz iteration for S^{-1/2} (Higham, Functions of Matrices, 2008, Sec. 6.3):
// Y0 = S/c, Z0 = I, T = (3I - Z Y)/2, Y <- Y T, Z <- T Z; Z -> (S/c)^{-1/2}, c = ||S||_F.
int newton_schulz_invsqrt(const double* S, double* Xout, double* Y, double* Z, double* T,
                          double* P, int n, int iters, cudaStream_t st, double* work, size_t work_cap) {
    long long nn = (long long)n * n;
    k_frob<<<1, 256, 0, st>>>(S, nn, T);
    NOF_LAUNCH_CHECK();
    double h_nrm = 0.0;
    NOF_CUDA(cudaMemcpyAsync(&h_nrm, T, sizeof(double), cudaMemcpyDeviceToHost, st));
    NOF_CUDA(cudaStreamSynchronize(st));
    if (!(h_nrm > 0.0) || !std::isfinite(h_nrm)) {
        nof_set_error("newton_schulz_invsqrt: overlap matrix has no finite positive norm");
        return NOF_ENONFINITE;
    }
    k_scale<<<blocks_for(nn), 256, 0, st>>>(S, 1.0 / h_nrm, Y, nn);
    NOF_LAUNCH_CHECK();
    k_axpy_identity<<<blocks_for(nn), 256, 0, st>>>(S, 0.0, Z, n);  // Z = I
    NOF_LAUNCH_CHECK();
    for (int it = 0; it < iters; ++it) {
        NOF_TRY(gemm64(square_gemm(Z, Y, P, n, work, work_cap), st));   // P = Z Y
        k_ns_mid<<<blocks_for(nn), 256, 0, st>>>(P, T, n);  // T = 1.5 I - 0.5 P
        NOF_LAUNCH_CHECK();
        NOF_TRY(gemm64(square_gemm(Y, T, P, n, work, work_cap), st));   // P = Y T
        double* tmp = Y; Y = P; P = tmp;
        NOF_TRY(gemm64(square_gemm(T, Z, P, n, work, work_cap), st));   // P = T Z
        tmp = Z; Z = P; P = tmp;
    }
    k_scale<<<blocks_for(nn), 256, 0, st>>>(Z, 1.0 / std::sqrt(h_nrm), Xout, nn);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

// U = exp(y) for antisymmetric y: s = smallest integer with ||y||_F / 2^s <= 1/2,
// Horner form of the degree-12 Taylor polynomial of z = y / 2^s, then s squarings.
// *flag |= NOF_DEV_RANGE when *nrm > limit (one thread)
__global__ void k_range_check(const double* nrm, double limit, int* flag) {
    if (!(*nrm <= limit)) atomicOr(flag, NOF_DEV_RANGE);
}

int expm_antisym_device_fixed(const double* y, double* U, double* w1, double* w2, int n, int* status,
                              cudaStream_t st, double* work, size_t work_cap) {
    constexpr int kS = 12;
    long long nn = (long long)n * n;
    k_frob<<<1, 256, 0, st>>>(y, nn, w1);
    NOF_LAUNCH_CHECK();
    k_range_check<<<1, 1, 0, st>>>(w1, std::ldexp(1.0, kS), status);
    NOF_LAUNCH_CHECK();
    double* z = w1;  // the norm is no longer needed
    k_scale<<<blocks_for(nn), 256, 0, st>>>(y, std::ldexp(1.0, -kS), z, nn);
    NOF_LAUNCH_CHECK();
    k_axpy_identity<<<blocks_for(nn), 256, 0, st>>>(z, 0.0, U, n);
    NOF_LAUNCH_CHECK();
    for (int k = 12; k >= 1; --k) {
        NOF_TRY(gemm64(square_gemm(z, U, w2, n, work, work_cap), st));  // w2 = z U
        k_axpy_identity<<<blocks_for(nn), 256, 0, st>>>(w2, 1.0 / k, U, n);
        NOF_LAUNCH_CHECK();
    }
    for (int i = 0; i < kS; ++i) {
        NOF_TRY(gemm64(square_gemm(U, U, w2, n, work, work_cap), st));
        NOF_CUDA(cudaMemcpyAsync(U, w2, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    return NOF_OK;
}

int expm_antisym_device(const double* y, double* U, double* w1, double* w2, int n,
                        cudaStream_t st, double* work, size_t work_cap) {
    long long nn = (long long)n * n;
    k_frob<<<1, 256, 0, st>>>(y, nn, w1);
    NOF_LAUNCH_CHECK();
    double h_nrm = 0.0;
    NOF_CUDA(cudaMemcpyAsync(&h_nrm, w1, sizeof(double), cudaMemcpyDeviceToHost, st));
    NOF_CUDA(cudaStreamSynchronize(st));
    int s = 0;
    while (h_nrm / std::ldexp(1.0, s) > 0.5) ++s;
    double* z = w1;
    k_scale<<<blocks_for(nn), 256, 0, st>>>(y, std::ldexp(1.0, -s), z, nn);
    NOF_LAUNCH_CHECK();
    // U = I
    k_axpy_identity<<<blocks_for(nn), 256, 0, st>>>(z, 0.0, U, n);
    NOF_LAUNCH_CHECK();
    for (int k = 12; k >= 1; --k) {
        NOF_TRY(gemm64(square_gemm(z, U, w2, n, work, work_cap), st));  // w2 = z U
        k_axpy_identity<<<blocks_for(nn), 256, 0, st>>>(w2, 1.0 / k, U, n);
        NOF_LAUNCH_CHECK();
    }
    for (int i = 0; i < s; ++i) {
        NOF_TRY(gemm64(square_gemm(U, U, w2, n, work, work_cap), st));
        NOF_CUDA(cudaMemcpyAsync(U, w2, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    return NOF_OK;
}
