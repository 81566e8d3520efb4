// Nuclear gradient of the RI-PNOF energy for s bases (FP64 path). C ABI: nof_nuclear_gradient.
//
// Along the orbital connection C(x) = C0 (C0^T S(x) C0)^{-1/2}, at any (C, gamma):
//   dE/dx = sum_uv P_uv h^x_uv - 2 sum_uv (C lambda C^T)_uv S^x_uv
//         + sum_P sum_uv Gamma^P_uv (uv|P)^x - sum_PQ Z_PQ V^x_PQ + V_nn^x,
// P = 2 C diag(n) C^T, c^P_pq = sum_Q (V^-1)_PQ (Q|pq) = (L^-T b)^P_pq,
// Y^P_pq = 2 delta_pq sum_r A_pr c^P_rr - 2 B_pq c^P_pq, Gamma^P = C Y^P C^T,
// Z_PQ = sum_pq (A_pq c^P_pp c^Q_qq - B_pq c^P_pq c^Q_pq).
// The integral derivatives (closed forms for s Gaussians) are evaluated on the fly. Every term is
// a sum over pairs or triples whose derivative with respect to a centre is collected per basis
// function, aux function or nucleus in fixed-order block reductions, then per atom (no atomics,
// so the result does not depend on scheduling). Derivatives with respect to the second centre of
// a symmetric pair equal those with respect to the first after swapping the pair, which gives the
// factors of 2 below; the aux centre of (uv|P) takes minus the sum of the other two.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi52 = 34.98683665524972497;  // 2 pi^{5/2}
// Screening: a primitive pair with mu |A-B|^2 > 39 has a Gaussian product exp(-mu |A-B|^2) below
// 1.2e-17, and every integral and derivative of it carries that factor; such pairs are skipped
// before any exponential is taken.
constexpr double kScreenExponent = 39.0;

__device__ __forceinline__ double g_boys0(double t) {
    if (t < 1e-8) return 1.0 - t / 3.0 + t * t / 10.0;
    const double st = sqrt(t);
    return 0.88622692545275801365 * erf(st) / st;
}
// F1(t) = -dF0/dt = int_0^1 u^2 exp(-t u^2) du
__device__ __forceinline__ double g_boys1(double t) {
    if (t < 1e-4) return 1.0 / 3.0 - t / 5.0 + t * t / 14.0;
    return (g_boys0(t) - exp(-t)) / (2.0 * t);
}
__device__ __forceinline__ double g_norm(double a) { return pow(2.0 * a / kPi, 0.75); }

// Fixed-order block reduction of three values (256 threads); thread 0 returns the sums.
__device__ void block_sum3(double v[3], double* red) {
    for (int k = 0; k < 3; ++k) red[k * 256 + threadIdx.x] = v[k];
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o)
            for (int k = 0; k < 3; ++k) red[k * 256 + threadIdx.x] += red[k * 256 + threadIdx.x + o];
        __syncthreads();
    }
    for (int k = 0; k < 3; ++k) v[k] = red[k * 256];
}

struct Basis {
    const int *fn_atom, *fn_first, *fn_nprim;
    const double *pexp, *pcoef, *xyz, *Z;
    int n, natom;
    const int* ax_atom;
    const double* axexp;
    int X;
};

// Y^P_pq = 2 delta_pq sum_r A_pr c^P_rr - 2 B_pq c^P_pq
__global__ void k_grad_Y(const double* cfit, const double* A, const double* Bc, int X, int a, double* Y) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long aa = (long long)a * a;
    if (i >= (long long)X * aa) return;
    const int P = (int)(i / aa), r = (int)(i - P * aa), p = r / a, q = r - p * a;
    const double* c = cfit + P * aa;
    double v = -2.0 * Bc[r] * c[r];
    if (p == q) {
        double s = 0.0;
        for (int t = 0; t < a; ++t) s += A[p * a + t] * c[(long long)t * a + t];
        v += 2.0 * s;
    }
    Y[i] = v;
}
__global__ void k_grad_cdiag(const double* cfit, int X, int a, double* cd) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)X * a) return;
    const int P = (int)(i / a), p = (int)(i - (long long)P * a);
    cd[i] = cfit[(long long)P * a * a + (long long)p * a + p];
}
__global__ void k_grad_hadamard(const double* Bc, const double* cfit, int X, int a, double* out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long aa = (long long)a * a;
    if (i >= (long long)X * aa) return;
    out[i] = Bc[i % aa] * cfit[i];
}
// out[u][p] = f occ[p] C[u][p] for p < a
__global__ void k_grad_scale_cols(const double* C, const double* occ, int n, int a, double f, double* out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)n * a) return;
    const int u = (int)(i / a), p = (int)(i - (long long)u * a);
    out[i] = f * occ[p] * C[(long long)u * n + p];
}

// F1[u] = sum_v [P_uv (dT + dV_basis)/dA_u - 2 Wsym_uv dS/dA_u] (A_u = centre of u)
__global__ void __launch_bounds__(256) k_grad_1e_rows(Basis bs, const double* Pao, const double* Wao, double* F1) {
    __shared__ double red[3 * 256];
    const int u = blockIdx.x, n = bs.n;
    const double* A = bs.xyz + 3 * bs.fn_atom[u];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int v = threadIdx.x; v < n; v += 256) {
        const double* B = bs.xyz + 3 * bs.fn_atom[v];
        const double AB[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]};
        const double ab2 = AB[0] * AB[0] + AB[1] * AB[1] + AB[2] * AB[2];
        const double Puv = Pao[(long long)u * n + v];
        const double Wuv = 0.5 * (Wao[(long long)u * n + v] + Wao[(long long)v * n + u]);
        for (int i = 0; i < bs.fn_nprim[u]; ++i) {
            const double a = bs.pexp[bs.fn_first[u] + i], ca = bs.pcoef[bs.fn_first[u] + i];
            for (int j = 0; j < bs.fn_nprim[v]; ++j) {
                const double b = bs.pexp[bs.fn_first[v] + j], cb = bs.pcoef[bs.fn_first[v] + j];
                const double p = a + b, mu = a * b / p;
                if (mu * ab2 > kScreenExponent) continue;
                const double K = exp(-mu * ab2), w = ca * cb;
                const double r = kPi / p;
                const double Sp = r * sqrt(r) * K;
                // overlap and kinetic: first-centre derivatives
                const double fS = -2.0 * mu * Sp, fT = -2.0 * mu * mu * (5.0 - 2.0 * mu * ab2) * Sp;
                for (int k = 0; k < 3; ++k) acc[k] += w * AB[k] * (Puv * fT - 2.0 * Wuv * fS);
                // nuclear attraction of every nucleus: first-centre derivative
                const double Pc[3] = {(a * A[0] + b * B[0]) / p, (a * A[1] + b * B[1]) / p, (a * A[2] + b * B[2]) / p};
                for (int C = 0; C < bs.natom; ++C) {
                    const double* R = bs.xyz + 3 * C;
                    const double PC[3] = {Pc[0] - R[0], Pc[1] - R[1], Pc[2] - R[2]};
                    const double t = p * (PC[0] * PC[0] + PC[1] * PC[1] + PC[2] * PC[2]);
                    const double pre = -bs.Z[C] * 2.0 * kPi / p;
                    const double F0 = g_boys0(t), F1v = g_boys1(t);
                    for (int k = 0; k < 3; ++k)
                        acc[k] += w * Puv * pre * (-2.0 * mu * AB[k] * K * F0 - 2.0 * a * K * F1v * PC[k]);
                }
            }
        }
    }
    block_sum3(acc, red);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) F1[3 * u + k] = acc[k];
}

// Gp[C][s] = sum over the pairs uv of slice s of P_uv dV^C_uv / dR_C (the operator centre);
// block (C, s), the pairs strided over gridDim.y slices.
__global__ void __launch_bounds__(256) k_grad_1e_ops(Basis bs, const double* Pao, double* Gp) {
    __shared__ double red[3 * 256];
    const int C = blockIdx.x, n = bs.n;
    const double* R = bs.xyz + 3 * C;
    double acc[3] = {0.0, 0.0, 0.0};
    for (long long uv = blockIdx.y * 256LL + threadIdx.x; uv < (long long)n * n; uv += 256LL * gridDim.y) {
        const int u = (int)(uv / n), v = (int)(uv - (long long)u * n);
        const double* A = bs.xyz + 3 * bs.fn_atom[u];
        const double* B = bs.xyz + 3 * bs.fn_atom[v];
        const double ab2 = (A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) + (A[2] - B[2]) * (A[2] - B[2]);
        const double Puv = Pao[uv];
        for (int i = 0; i < bs.fn_nprim[u]; ++i) {
            const double a = bs.pexp[bs.fn_first[u] + i], ca = bs.pcoef[bs.fn_first[u] + i];
            for (int j = 0; j < bs.fn_nprim[v]; ++j) {
                const double b = bs.pexp[bs.fn_first[v] + j], cb = bs.pcoef[bs.fn_first[v] + j];
                const double p = a + b;
                if (a * b / p * ab2 > kScreenExponent) continue;
                const double K = exp(-a * b / p * ab2);
                const double PC[3] = {(a * A[0] + b * B[0]) / p - R[0], (a * A[1] + b * B[1]) / p - R[1],
                                      (a * A[2] + b * B[2]) / p - R[2]};
                const double t = p * (PC[0] * PC[0] + PC[1] * PC[1] + PC[2] * PC[2]);
                const double f = ca * cb * Puv * (-bs.Z[C] * 2.0 * kPi / p) * 2.0 * p * K * g_boys1(t);
                for (int k = 0; k < 3; ++k) acc[k] += f * PC[k];
            }
        }
    }
    block_sum3(acc, red);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) Gp[((long long)C * gridDim.y + blockIdx.y) * 3 + k] = acc[k];
}

// One primitive pair of (uv|P): accumulate the first-centre derivative (w.r.t. A_u) into d1 and
// the aux-centre derivative into dP, each weighted by g.
__device__ __forceinline__ void three_center_pair(double a, double b, double w, const double* A, const double* B,
                                                  const double* Cc, double q, double nq, double g, double d1[3],
                                                  double dP[3]) {
    const double p = a + b, mu = a * b / p;
    const double AB[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]};
    const double mab2 = mu * (AB[0] * AB[0] + AB[1] * AB[1] + AB[2] * AB[2]);
    if (mab2 > kScreenExponent) return;
    const double K = exp(-mab2);
    const double PC[3] = {(a * A[0] + b * B[0]) / p - Cc[0], (a * A[1] + b * B[1]) / p - Cc[1],
                          (a * A[2] + b * B[2]) / p - Cc[2]};
    const double rho = p * q / (p + q);
    const double t = rho * (PC[0] * PC[0] + PC[1] * PC[1] + PC[2] * PC[2]);
    const double pre = g * w * nq * kTwoPi52 / (p * q * sqrt(p + q));
    const double F0 = g_boys0(t), F1v = g_boys1(t);
    for (int k = 0; k < 3; ++k) {
        d1[k] += pre * (-2.0 * mu * AB[k] * K * F0 - 2.0 * rho * (a / p) * K * F1v * PC[k]);
        dP[k] += pre * 2.0 * rho * K * F1v * PC[k];
    }
}

// One pass over the triples (u, v, P): block (u, chunk) takes basis function u and the aux
// functions P of its chunk of 256, one per thread. F3p[u][chunk] = sum_v sum_P Gamma^P_uv
// d(uv|P)/dA_u (fixed-order block sum) and HPu[u][P] = sum_v Gamma^P_uv d(uv|P)/dR_P (one
// thread per P, so no reduction is needed); the sums over chunks and over u follow in order.
__global__ void __launch_bounds__(256) k_grad_3c(Basis bs, const double* Gam, double* F3p, double* HPu) {
    __shared__ double red[3 * 256];
    const int u = blockIdx.x, n = bs.n, X = bs.X;
    const double* A = bs.xyz + 3 * bs.fn_atom[u];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int P = blockIdx.y * 256 + threadIdx.x; P < X && P < (int)(blockIdx.y + 1) * 256; P += 256) {
        const double* Cc = bs.xyz + 3 * bs.ax_atom[P];
        const double q = bs.axexp[P], nq = g_norm(q);
        double dP[3] = {0.0, 0.0, 0.0};
        for (int v = 0; v < n; ++v) {
            const double g = Gam[((long long)P * n + u) * n + v];
            const double* B = bs.xyz + 3 * bs.fn_atom[v];
            for (int i = 0; i < bs.fn_nprim[u]; ++i)
                for (int j = 0; j < bs.fn_nprim[v]; ++j)
                    three_center_pair(bs.pexp[bs.fn_first[u] + i], bs.pexp[bs.fn_first[v] + j],
                                      bs.pcoef[bs.fn_first[u] + i] * bs.pcoef[bs.fn_first[v] + j], A, B, Cc, q, nq, g,
                                      acc, dP);
        }
        for (int k = 0; k < 3; ++k) HPu[((long long)u * X + P) * 3 + k] = dP[k];
    }
    block_sum3(acc, red);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) F3p[((long long)u * gridDim.y + blockIdx.y) * 3 + k] = acc[k];
}

// HP[P] = sum_u HPu[u][P] in order of u; F3[u] = sum_c F3p[u][c] in order of c
__global__ void k_grad_3c_sums(const double* HPu, const double* F3p, int n, int X, int nch, double* HP,
                               double* F3) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < 3LL * X) {
        double s = 0.0;
        for (int u = 0; u < n; ++u) s += HPu[(long long)u * 3 * X + i];
        HP[i] = s;
    } else if (i < 3LL * X + 3LL * n) {
        const long long j = i - 3LL * X;
        const int u = (int)(j / 3), k = (int)(j % 3);
        double s = 0.0;
        for (int c = 0; c < nch; ++c) s += F3p[((long long)u * nch + c) * 3 + k];
        F3[j] = s;
    }
}

// E2[P] = sum_Q Z_PQ d(P|Q)/dR_P
__global__ void __launch_bounds__(256) k_grad_2c_rows(Basis bs, const double* Zm, double* E2) {
    __shared__ double red[3 * 256];
    const int P = blockIdx.x, X = bs.X;
    const double* Cp = bs.xyz + 3 * bs.ax_atom[P];
    const double p = bs.axexp[P], np_ = g_norm(p);
    double acc[3] = {0.0, 0.0, 0.0};
    for (int Q = threadIdx.x; Q < X; Q += 256) {
        const double* Cq = bs.xyz + 3 * bs.ax_atom[Q];
        const double q = bs.axexp[Q];
        const double D[3] = {Cp[0] - Cq[0], Cp[1] - Cq[1], Cp[2] - Cq[2]};
        const double rho = p * q / (p + q);
        const double t = rho * (D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
        const double f = -Zm[(long long)P * X + Q] * np_ * g_norm(q) * kTwoPi52 / (p * q * sqrt(p + q)) *
                         2.0 * rho * g_boys1(t);
        for (int k = 0; k < 3; ++k) acc[k] += f * D[k];
    }
    block_sum3(acc, red);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) E2[3 * P + k] = acc[k];
}

// grad[A] = 2 sum_{u on A} (F1 + F3)[u] + G[A] + sum_{P on A} (HP - 2 E2)[P] + dV_nn/dR_A
__global__ void k_grad_assemble(Basis bs, const double* F1, const double* F3, const double* Gp, int nslice,
                                const double* HP, const double* E2, double* grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * bs.natom) return;
    const int A = i / 3, k = i - 3 * A;
    double s = 0.0;
    for (int u = 0; u < bs.n; ++u)
        if (bs.fn_atom[u] == A) s += 2.0 * (F1[3 * u + k] + F3[3 * u + k]);
    for (int sl = 0; sl < nslice; ++sl) s += Gp[((long long)A * nslice + sl) * 3 + k];
    for (int P = 0; P < bs.X; ++P)
        if (bs.ax_atom[P] == A) s += HP[3 * P + k] - 2.0 * E2[3 * P + k];
    const double* RA = bs.xyz + 3 * A;
    for (int B = 0; B < bs.natom; ++B) {
        if (B == A) continue;
        const double* RB = bs.xyz + 3 * B;
        const double d0 = RA[0] - RB[0], d1 = RA[1] - RB[1], d2 = RA[2] - RB[2];
        const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        const double dk = k == 0 ? d0 : (k == 1 ? d1 : d2);
        s -= bs.Z[A] * bs.Z[B] * dk / (r * r * r);
    }
    grad[i] = s;
}

inline unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

template <class T>
int galloc(T** p, size_t count) {
    if (*p) return NOF_OK;
    cudaError_t e = cudaMalloc((void**)p, (count ? count : 1) * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return nof_cuda_fail(e, "cudaMalloc (nuclear gradient workspaces)", __FILE__, __LINE__);
    }
    return NOF_OK;
}

Gemm64 mk(int M, int N, int K, const double* A, long long sAm, long long sAk0, const double* B, long long sBn,
          long long sBk0, double* C, long long sCm, nof_ctx* c) {
    Gemm64 g;
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.sAm = sAm; g.sAk0 = sAk0;
    g.B = B; g.sBn = sBn; g.sBk0 = sBk0;
    g.C = C; g.sCm = sCm; g.sCn = 1;
    g.work = c->gwork; g.work_cap = c->gwork_cap;
    return g;
}

}  // namespace

extern "C" int nof_nuclear_gradient(nof_ctx* c, const double* C, const double* gamma, double* grad) {
    if (!c) {
        nof_set_error("null context");
        return NOF_EINVAL;
    }
    if (!c->built) {
        nof_set_error("nof_build_B has not been called on this context");
        return NOF_ESTATE;
    }
    if (!C || !gamma || !grad) {
        nof_set_error("nof_nuclear_gradient: null pointer");
        return NOF_EINVAL;
    }
    if (c->opt.precision != NOF_PREC_FP64 || !c->Linv) {
        nof_set_error("nof_nuclear_gradient: needs a NOF_PREC_FP64 context");
        return NOF_EINVAL;
    }
    const int n = c->nbf, X = c->naux, a = c->nact, natom = c->natom;
    const long long aa = (long long)a * a, nn = (long long)n * n;
    cudaStream_t st = c->stream;
    NOF_TRY(plain_jk(c, C));
    NOF_TRY(plain_grad(c, C, gamma, true));  // b, A, B, occupations, lambda
    NOF_TRY(galloc(&c->gr_cfit, (size_t)(X * aa)));
    NOF_TRY(galloc(&c->gr_Y, (size_t)(X * aa)));
    NOF_TRY(galloc(&c->gr_Gam, (size_t)(X * nn)));
    NOF_TRY(galloc(&c->gr_Z, (size_t)X * X));
    const int nch = (X + 255) / 256;
    const int nslice = (int)std::min<long long>(32, (nn + 4095) / 4096);
    NOF_TRY(galloc(&c->gr_small, (size_t)(2 * X * a + 3 * nn + 3 * (2 * n + 2 * X) + 3LL * n * X + 3LL * n * nch +
                                          3LL * natom * 32)));
    double* cd = c->gr_small;
    double* tXa = cd + (long long)X * a;
    double* Pao = tXa + (long long)X * a;
    double* Wao = Pao + nn;
    double* tn = Wao + nn;
    double* F1 = tn + nn;
    double* F3 = F1 + 3 * n;
    double* HP = F3 + 3 * n;
    double* E2 = HP + 3 * X;
    double* HPu = E2 + 3 * X;              // [n][X][3]
    double* F3p = HPu + 3LL * n * X;       // [n][nch][3]
    double* G = F3p + 3LL * n * nch;       // [natom][nslice][3]
    // fitting coefficients c = L^-T b
    {
        Gemm64 g = mk(X, (int)aa, X, c->Linv, 1, X, c->b, 1, aa, c->gr_cfit, aa, c);
        NOF_TRY(gemm64(g, st));
    }
    k_grad_Y<<<blocks(X * aa), 256, 0, st>>>(c->gr_cfit, c->A, c->Bc, X, a, c->gr_Y);
    NOF_LAUNCH_CHECK();
    {   // Gamma^P = C_a Y^P C_a^T through T (X n a) as scratch
        Gemm64 g = mk(n, a, a, C, n, 1, c->gr_Y, 1, a, c->T, a, c);
        g.batch = X; g.bB = aa; g.bC = (long long)n * a;
        NOF_TRY(gemm64(g, st));
        Gemm64 h = mk(n, n, a, c->T, a, 1, C, n, 1, c->gr_Gam, n, c);
        h.batch = X; h.bA = (long long)n * a; h.bC = nn;
        NOF_TRY(gemm64(h, st));
    }
    // Z = cdiag A cdiag^T - (B o c) c^T
    k_grad_cdiag<<<blocks((long long)X * a), 256, 0, st>>>(c->gr_cfit, X, a, cd);
    NOF_LAUNCH_CHECK();
    NOF_TRY(gemm64(mk(X, a, a, cd, a, 1, c->A, 1, a, tXa, a, c), st));
    NOF_TRY(gemm64(mk(X, X, a, tXa, a, 1, cd, a, 1, c->gr_Z, X, c), st));
    k_grad_hadamard<<<blocks(X * aa), 256, 0, st>>>(c->Bc, c->gr_cfit, X, a, c->gr_Y);
    NOF_LAUNCH_CHECK();
    {
        Gemm64 g = mk(X, X, (int)aa, c->gr_Y, aa, 1, c->gr_cfit, aa, 1, c->gr_Z, X, c);
        g.alpha = -1.0; g.beta = 1.0;
        NOF_TRY(gemm64(g, st));
    }
    // P = 2 C_a diag(n) C_a^T; W = C lambda_a C_a^T
    k_grad_scale_cols<<<blocks((long long)n * a), 256, 0, st>>>(C, c->occ, n, a, 2.0, tn);
    NOF_LAUNCH_CHECK();
    NOF_TRY(gemm64(mk(n, n, a, tn, a, 1, C, n, 1, Pao, n, c), st));
    NOF_TRY(gemm64(mk(n, a, n, C, n, 1, c->lam, 1, n, tn, a, c), st));
    NOF_TRY(gemm64(mk(n, n, a, tn, a, 1, C, n, 1, Wao, n, c), st));
    Basis bs{c->fn_atom, c->fn_first, c->fn_nprim, c->pexp, c->pcoef, c->xyz, c->Z, n, natom, c->ax_atom, c->axexp, X};
    k_grad_1e_rows<<<n, 256, 0, st>>>(bs, Pao, Wao, F1);
    NOF_LAUNCH_CHECK();
    k_grad_1e_ops<<<dim3(natom, nslice), 256, 0, st>>>(bs, Pao, G);
    NOF_LAUNCH_CHECK();
    k_grad_3c<<<dim3(n, nch), 256, 0, st>>>(bs, c->gr_Gam, F3p, HPu);
    NOF_LAUNCH_CHECK();
    k_grad_3c_sums<<<blocks(3LL * (X + n)), 256, 0, st>>>(HPu, F3p, n, X, nch, HP, F3);
    NOF_LAUNCH_CHECK();
    k_grad_2c_rows<<<X, 256, 0, st>>>(bs, c->gr_Z, E2);
    NOF_LAUNCH_CHECK();
    k_grad_assemble<<<blocks(3 * natom, 128), 128, 0, st>>>(bs, F1, F3, G, nslice, HP, E2, grad);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}
