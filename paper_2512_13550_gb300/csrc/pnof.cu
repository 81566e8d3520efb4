// PNOF pairing-coefficient, energy, Lagrangian and gradient kernels (FP64) and the plain FP64
// evaluation path.
//
// Occupations: trigonometric mapping (Occupation Number Optimization subsection):
//   n_g = (1 + cos^2 gamma_g)/2, h_g = 1 - n_g,
//   n_{p_i} = h_g cos^2 gamma_{p_1} ... cos^2 gamma_{p_{i-1}} sin^2 gamma_{p_i} (i < N_g),
//   n_{p_{N_g}} = h_g cos^2 gamma_{p_1} ... cos^2 gamma_{p_{N_g - 1}},
// which keeps the sum rule of Eq. sum1. sqrt(n) and sqrt(1 - n) are formed from |sin|, |cos|
// so their gamma-derivatives never divide by a vanishing occupation (one-sided at gamma = 0).
// Energy: Eq. PNOF, E = 2 sum n_p h_pp + sum A_pq J_pq - sum B_pq K_pq + V_nn, with the
// spin-restricted PNOF7 coefficients: A_pp = n_p, A_pq = 2 n_p n_q (different subspaces);
// B_pq = -c_p c_q (same subspace, p != q; c = +sqrt n strong, -sqrt n weak),
// B_pq = n_p n_q + Phi_p Phi_q (different subspaces; PNOF5 drops Phi), Phi = sqrt(n(1-n)).
// Lagrangian (Natural Orbital Optimization subsection): lambda = C^T Lambda,
//   Lambda_mu,p = n_p (HC)_mu,p + sum_P sum_r T^P_mu,r W^P_rp,
//   W^P_rp = delta_rp D^P_p - B_pr b^P_rp,  D^P = A d^P,
// and g = 4 (lambda - lambda^T).
#include <cmath>

#include "internal.h"

namespace {

inline unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ double sgn1(double x) { return x >= 0.0 ? 1.0 : -1.0; }

// One thread per subspace g: s = sqrt(n), t = sqrt(1-n) and their derivatives with respect to
// the N_g angles of the subspace (ds[p * ncwo + slot]).
__device__ void occupations_trig(int g, const double* gamma, int npair, int ncwo, double* s, double* t, double* ds,
                                 double* dt) {    const double rt2 = 1.4142135623730950488;
    double th0 = gamma[g];
    double s0 = sin(th0), c0 = cos(th0);
    double sg = sqrt(0.5 * (1.0 + c0 * c0));
    double tg = fabs(s0) / rt2;
    double dsg = (-s0 * c0) / (2.0 * sg);
    double dtg = sgn1(s0) * c0 / rt2;
    s[g] = sg;
    t[g] = tg;
    for (int k = 0; k < ncwo; ++k) {
        ds[g * ncwo + k] = (k == 0) ? dsg : 0.0;
        dt[g * ncwo + k] = (k == 0) ? dtg : 0.0;
    }
    for (int i = 1; i <= ncwo; ++i) {
        int p = npair + (i - 1) * npair + (npair - 1 - g);
        // factors: slot 0 -> tg; slots 1..i-1 -> |cos|; slot i (if i < ncwo) -> |sin|
        double val = tg;
        for (int j = 1; j < i; ++j) val *= fabs(cos(gamma[j * npair + g]));
        if (i < ncwo) val *= fabs(sin(gamma[i * npair + g]));
        for (int k = 0; k < ncwo; ++k) {
            double d = 0.0;
            // derivative of factor k times the product of the others
            bool has = (k == 0) || (k < i) || (k == i && i < ncwo);
            if (has) {
                double dk, prod = 1.0;
                if (k == 0) dk = dtg; else prod = tg;
                for (int j = 1; j < i; ++j) {
                    double th = gamma[j * npair + g];
                    if (j == k) dk = -sgn1(cos(th)) * sin(th);
                    else prod *= fabs(cos(th));
                }
                if (i < ncwo) {
                    double th = gamma[i * npair + g];
                    if (k == i) dk = sgn1(sin(th)) * cos(th);
                    else prod *= fabs(sin(th));
                }
                d = dk * prod;
            }
            ds[p * ncwo + k] = d;
        }
        double tp = sqrt(1.0 - val * val);
        s[p] = val;
        t[p] = tp;
        for (int k = 0; k < ncwo; ++k) dt[p * ncwo + k] = -val * ds[p * ncwo + k] / tp;
    }
}

__global__ void k_occupations(const double* gamma, int npair, int ncwo, double* s, double* t,
                              double* ds, double* dt) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= npair) return;
    occupations_trig(g, gamma, npair, ncwo, s, t, ds, dt);
}

// Softmax mapping (isoftmax = 1), same outputs as k_occupations. Subspace g has the variables
// x_k = gamma[k * npair + g] (k < ncwo), x_k belonging to the weak orbital p_{k+1}:
//   Z = 1 + sum_k exp(x_k),  n_g = 1 / Z,  n_{p_i} = exp(x_{i-1}) / Z,
//   d sqrt(n_q) / d x_k = sqrt(n_q) ([q = p_{k+1}] - n_{p_{k+1}}) / 2,
//   d sqrt(1 - n_q) = -sqrt(n_q) d sqrt(n_q) / sqrt(1 - n_q).
// The exponentials are taken relative to max(0, max_k x_k) so that none overflows, and 1 - n_q
// is summed from the other orbitals' weights (no cancellation).
__device__ void occupations_softmax(int g, const double* gamma, int npair, int ncwo, double* s, double* t,
                                    double* ds, double* dt) {    double m = 0.0;
    for (int k = 0; k < ncwo; ++k) m = fmax(m, gamma[k * npair + g]);
    const double w0 = exp(-m);  // weight of the strong orbital, exp(0 - m)
    double z = w0;
    for (int k = 0; k < ncwo; ++k) z += exp(gamma[k * npair + g] - m);
    for (int q = 0; q <= ncwo; ++q) {  // q = 0: the strong orbital g; q = i: the weak orbital p_i
        const int p = q == 0 ? g : npair + (q - 1) * npair + (npair - 1 - g);
        const double w = q == 0 ? w0 : exp(gamma[(q - 1) * npair + g] - m);
        double rest = q == 0 ? 0.0 : w0;
        for (int k = 0; k < ncwo; ++k)
            if (k + 1 != q) rest += exp(gamma[k * npair + g] - m);
        const double sp = sqrt(w / z), tp = sqrt(rest / z);
        s[p] = sp;
        t[p] = tp;
        for (int k = 0; k < ncwo; ++k) {
            const double nk = exp(gamma[k * npair + g] - m) / z;
            const double d = 0.5 * sp * ((q == k + 1 ? 1.0 : 0.0) - nk);
            ds[p * ncwo + k] = d;
            dt[p * ncwo + k] = -sp * d / tp;
        }
    }
}

__global__ void k_occupations_softmax(const double* gamma, int npair, int ncwo, double* s, double* t,
                                      double* ds, double* dt) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= npair) return;
    occupations_softmax(g, gamma, npair, ncwo, s, t, ds, dt);
}

// A and B of Eq. PNOF for every active pair (p, q); optionally also as double-floats (hi, lo) for
// the split path (Adf, Bcdf may be null).
__device__ void coefficient_one(long long idx, const double* s, const double* t, const int* pair, const int* slot,
                                int a, int ipnof, double* occ, double* A, double* Bc, float2* Adf, float2* Bcdf) {    int p = (int)(idx / a), q = (int)(idx % a);
    double np = s[p] * s[p], nq = s[q] * s[q];
    if (q == 0) occ[p] = np;
    double av, bv;
    if (p == q) {
        av = np;
        bv = 0.0;
    } else if (pair[p] == pair[q]) {
        double cp = slot[p] == 0 ? s[p] : -s[p];
        double cq = slot[q] == 0 ? s[q] : -s[q];
        av = 0.0;
        bv = -cp * cq;
    } else {
        av = 2.0 * np * nq;
        bv = np * nq;
        if (ipnof == 7) bv += (s[p] * t[p]) * (s[q] * t[q]);
    }
    A[idx] = av;
    Bc[idx] = bv;
    if (Adf) {
        const float ah = (float)av, bh = (float)bv;
        Adf[idx] = make_float2(ah, (float)(av - (double)ah));
        Bcdf[idx] = make_float2(bh, (float)(bv - (double)bh));
    }
}

__global__ void k_coefficients(const double* s, const double* t, const int* pair, const int* slot,
                               int a, int ipnof, double* occ, double* A, double* Bc, float2* Adf,
                               float2* Bcdf) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)a * a) return;
    coefficient_one(idx, s, t, pair, slot, a, ipnof, occ, A, Bc, Adf, Bcdf);
}

// hpp_p = sum_mu C_mu,p (H C)_mu,p, one warp per p
__global__ void k_hpp(const double* C, const double* HC, int n, int a, double* hpp) {
    int p = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (p >= a) return;
    double s = 0.0;
    for (int mu = lane; mu < n; mu += 32) s = fma(C[(long long)mu * n + p], HC[(long long)mu * a + p], s);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) hpp[p] = s;
}

// d^P_p = b^P_pp
__global__ void k_diag(const double* b, int X, int a, double* d) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)X * a) return;
    long long P = idx / a;
    int p = (int)(idx % a);
    d[idx] = b[P * a * a + (long long)p * a + p];
}

// K_pq = sum_P (b^P_pq)^2
__global__ void k_ksum(const double* b, int X, int a, double* K) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long aa = (long long)a * a;
    if (idx >= aa) return;
    double s = 0.0;
    for (int P = 0; P < X; ++P) {
        double v = b[P * aa + idx];
        s = fma(v, v, s);
    }
    K[idx] = s;
}

// W^P_rp = delta_rp D^P_p - B_pr b^P_rp
__global__ void k_build_W(const double* b, const double* D, const double* Bc, int X, int a,
                          double* W) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long aa = (long long)a * a;
    if (idx >= (long long)X * aa) return;
    long long P = idx / aa;
    long long rp = idx - P * aa;
    int r = (int)(rp / a), p = (int)(rp % a);
    double w = -Bc[(long long)p * a + r] * b[idx];
    if (r == p) w += D[P * a + p];
    W[idx] = w;
}

// Lambda = n_p HC + Lam' (in place in Lam)
__global__ void k_lambda_assemble(const double* HC, const double* occ, int n, int a, double* Lam) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n * a) return;
    int p = (int)(idx % a);
    Lam[idx] += occ[p] * HC[idx];
}

// g = 4 (lambda - lambda^T); lambda holds columns p < a (the others are zero and never stored).
// lambda = sum over the K split of the partial products work[split][n][a] (in split order, as
// gemm64 sums them) into lam (columns p < a, leading dimension n), and the orbital gradient
// g_pq = 4 (lambda_pq - lambda_qp) from the same sums, in one pass.
__global__ void k_reduce_gradient(const double* work, int splits, int n, int a, double* lam, double* g) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const int p = (int)(idx / n), q = (int)(idx % n);
    const long long MN = (long long)n * a;
    double lpq = 0.0, lqp = 0.0;
    if (q < a) {
        for (int s = 0; s < splits; ++s) lpq += work[s * MN + (long long)p * a + q];
        lam[idx] = lpq;
    }
    if (p < a)
        for (int s = 0; s < splits; ++s) lqp += work[s * MN + (long long)q * a + p];
    g[idx] = 4.0 * (lpq - lqp);
}

__global__ void k_orbital_gradient(const double* lam, int n, int a, double* g) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    int p = (int)(idx / n), q = (int)(idx % n);
    const double lpq = q < a ? lam[idx] : 0.0, lqp = p < a ? lam[(long long)q * n + p] : 0.0;
    g[idx] = 4.0 * (lpq - lqp);
}

// Partial derivatives of E with respect to n_p, c_p and Phi_p, and the energy row
// E_p = 2 n_p h_pp + sum_q (A_pq J_pq - B_pq K_pq), one warp per active orbital p
// (out [4][a]: dE/dn, dE/dc, dE/dPhi, E_p).
__device__ void dE_parts_warp(int p, int lane, const double* s, const double* t, const int* pair, const int* slot,
                              const double* hpp, const double* J, const double* K, const double* A,
                              const double* Bc, int a, int ipnof, double* out) {    double sn = 0.0, sc = 0.0, sf = 0.0, se = 0.0;
    for (int q = lane; q < a; q += 32) {
        const long long pq = (long long)p * a + q;
        double Jpq = J[pq], Kpq = K[pq];
        se += A[pq] * Jpq - Bc[pq] * Kpq;
        if (pair[q] != pair[p]) {
            double nq = s[q] * s[q];
            sn += nq * (2.0 * Jpq - Kpq);
            sf += (s[q] * t[q]) * Kpq;
        } else if (q != p) {
            double cq = slot[q] == 0 ? s[q] : -s[q];
            sc += cq * Kpq;
        }
    }
    for (int o = 16; o; o >>= 1) {
        sn += __shfl_xor_sync(0xffffffffu, sn, o);
        sc += __shfl_xor_sync(0xffffffffu, sc, o);
        sf += __shfl_xor_sync(0xffffffffu, sf, o);
        se += __shfl_xor_sync(0xffffffffu, se, o);
    }
    if (lane == 0) {
        out[p] = 2.0 * hpp[p] + J[(long long)p * a + p] + 2.0 * sn;
        out[a + p] = 2.0 * sc;
        out[2 * a + p] = (ipnof == 7) ? -2.0 * sf : 0.0;
        out[3 * a + p] = 2.0 * s[p] * s[p] * hpp[p] + se;
    }
}

__global__ void k_dE_parts(const double* s, const double* t, const int* pair, const int* slot,
                           const double* hpp, const double* J, const double* K, const double* A,
                           const double* Bc, int a, int ipnof, double* out) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= a) return;
    int p = warp;
    dE_parts_warp(p, lane, s, t, pair, slot, hpp, J, K, A, Bc, a, ipnof, out);
}

// dE/dgamma for gamma index k = i * npair + g: sum over the orbitals of subspace g. Warp 0 of
// block 0 also forms E = V_nn + sum_p E_p in a fixed order.
// dE/dgamma_k by the chain rule through sqrt(n), c and Phi of the orbitals of its subspace.
__device__ double gamma_chain_one(int k, const double* s, const double* t, const double* ds, const double* dt,
                                  const int* slot, const double* parts, int npair, int ncwo, int a) {
    int i = k / npair, g = k % npair;
    double acc = 0.0;
    for (int m = 0; m <= ncwo; ++m) {
        int p = (m == 0) ? g : npair + (m - 1) * npair + (npair - 1 - g);
        double dsk = ds[p * ncwo + i], dtk = dt[p * ncwo + i];
        double sign = slot[p] == 0 ? 1.0 : -1.0;
        acc += parts[p] * 2.0 * s[p] * dsk + parts[a + p] * sign * dsk +
               parts[2 * a + p] * (dsk * t[p] + s[p] * dtk);
    }
    return acc;
}

__global__ void k_gamma_chain(const double* s, const double* t, const double* ds, const double* dt,
                              const int* slot, const double* parts, int npair, int ncwo, int a,
                              const double* vnn, double* E, double* out, int* status) {
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        double e = 0.0;
        for (int p = threadIdx.x; p < a; p += 32) e += parts[3 * a + p];
        for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if (threadIdx.x == 0) {
            *E = e + *vnn;
            // a NaN or Inf in C, gamma or any stage before reaches the energy: flag it for nof_sync
            if (!isfinite(e)) atomicOr(status, NOF_DEV_NONFINITE);
        }
    }
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npair * ncwo) return;
    out[k] = gamma_chain_one(k, s, t, ds, dt, slot, parts, npair, ncwo, a);
}

// The ON update of nof_step (`iters` steepest-descent steps on gamma with J, K and h_pp fixed)
// in one block for systems with a <= 256: each iteration runs the occupations, the coefficients,
// the energy parts, the chain rule and the descent through the same device functions as the
// separate kernels, with block barriers between them, so the results are the same bits as those
// of the launch-per-kernel loop in a single launch instead of five per iteration.
__global__ void __launch_bounds__(1024) k_on_update_fused(double* gamma, int npair, int ncwo, int isoftmax,
                                                         double* s, double* t, double* ds, double* dt,
                                                         const int* pair, const int* slot, int a, int ipnof,
                                                         double* occ, double* A, double* Bc, float2* Adf,
                                                         float2* Bcdf, const double* hpp, const double* J,
                                                         const double* K, double* parts, double* ggam,
                                                         double lr, int iters) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    const int ng = npair * ncwo;
    for (int it = 0; it < iters; ++it) {
        for (int g = tid; g < npair; g += blockDim.x) {
            if (isoftmax) occupations_softmax(g, gamma, npair, ncwo, s, t, ds, dt);
            else occupations_trig(g, gamma, npair, ncwo, s, t, ds, dt);
        }
        __syncthreads();
        for (long long idx = tid; idx < (long long)a * a; idx += blockDim.x)
            coefficient_one(idx, s, t, pair, slot, a, ipnof, occ, A, Bc, Adf, Bcdf);
        __syncthreads();
        for (int p = warp; p < a; p += nw) dE_parts_warp(p, lane, s, t, pair, slot, hpp, J, K, A, Bc, a, ipnof, parts);
        __syncthreads();
        for (int k = tid; k < ng; k += blockDim.x) ggam[k] = gamma_chain_one(k, s, t, ds, dt, slot, parts, npair, ncwo, a);
        __syncthreads();
        for (int k = tid; k < ng; k += blockDim.x) gamma[k] -= lr * ggam[k];
        __syncthreads();
    }
}

// ---- ONs converged at fixed J, K, h_pp (the converged loop's first step) ------------------------
// Deterministic block reduction: every thread contributes its partial, shared memory sums them in a
// fixed tree; the result is returned to every thread.
__device__ double block_sum(double v, double* red) {
    const int tid = threadIdx.x;
    red[tid] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}
__device__ double block_max(double v, double* red) {
    const int tid = threadIdx.x;
    red[tid] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (tid < o) red[tid] = fmax(red[tid], red[tid + o]);
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// Energy row and partial derivatives of orbital p (as dE_parts_warp) with A and B formed on the fly
// from s = sqrt(n) and t = sqrt(1 - n) instead of read from the coefficient arrays.
__device__ void on_parts_warp(int p, int lane, const double* s, const double* t, const int* pair, const int* slot,
                              const double* hpp, const double* J, const double* K, int a, int ipnof, double* out) {
    const double np = s[p] * s[p], cp = slot[p] == 0 ? s[p] : -s[p], fp = s[p] * t[p];
    double sn = 0.0, sc = 0.0, sf = 0.0, se = 0.0;
    for (int q = lane; q < a; q += 32) {
        const long long pq = (long long)p * a + q;
        const double Jpq = J[pq], Kpq = K[pq];
        const double nq = s[q] * s[q];
        if (q == p) {
            se += np * Jpq;
        } else if (pair[q] != pair[p]) {
            const double fq = s[q] * t[q];
            const double bv = np * nq + (ipnof == 7 ? fp * fq : 0.0);
            se += 2.0 * np * nq * Jpq - bv * Kpq;
            sn += nq * (2.0 * Jpq - Kpq);
            sf += fq * Kpq;
        } else {
            const double cq = slot[q] == 0 ? s[q] : -s[q];
            se += cp * cq * Kpq;
            sc += cq * Kpq;
        }
    }
    for (int o = 16; o; o >>= 1) {
        sn += __shfl_xor_sync(0xffffffffu, sn, o);
        sc += __shfl_xor_sync(0xffffffffu, sc, o);
        sf += __shfl_xor_sync(0xffffffffu, sf, o);
        se += __shfl_xor_sync(0xffffffffu, se, o);
    }
    if (lane == 0) {
        out[p] = 2.0 * hpp[p] + J[(long long)p * a + p] + 2.0 * sn;
        out[a + p] = 2.0 * sc;
        out[2 * a + p] = (ipnof == 7) ? -2.0 * sf : 0.0;
        out[3 * a + p] = 2.0 * np * hpp[p] + se;
    }
}

// E(x) (without V_nn) and dE/dgamma at x into grad, by the whole block; returns E to every thread.
__device__ double on_eval_block(const double* x, double* grad, int npair, int ncwo, int isoftmax, double* s,
                                double* t, double* ds, double* dt, const int* pair, const int* slot, int a, int ipnof,
                                const double* hpp, const double* J, const double* K, double* parts, double* red) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    for (int g = tid; g < npair; g += blockDim.x) {
        if (isoftmax) occupations_softmax(g, x, npair, ncwo, s, t, ds, dt);
        else occupations_trig(g, x, npair, ncwo, s, t, ds, dt);
    }
    __syncthreads();
    for (int p = warp; p < a; p += nw) on_parts_warp(p, lane, s, t, pair, slot, hpp, J, K, a, ipnof, parts);
    __syncthreads();
    for (int k = tid; k < npair * ncwo; k += blockDim.x)
        grad[k] = gamma_chain_one(k, s, t, ds, dt, slot, parts, npair, ncwo, a);
    double e = 0.0;
    for (int p = tid; p < a; p += blockDim.x) e += parts[3 * a + p];
    return block_sum(e, red);  // its barriers also publish grad
}

// ONs optimised at fixed J, K, h_pp by BFGS with an Armijo step control, in one block (the
// algorithm and its constants are the oracle's: see oracle/optimize.py, on_converge). gamma is
// updated in place; w holds 6 ng + ng^2 doubles (trial point, gradients, s, y, H y, H);
// info[0] = accepted steps, info[1] = max |dE/dgamma| at the end (doubles).
__global__ void __launch_bounds__(1024) k_on_bfgs(double* gamma, int npair, int ncwo, int isoftmax, double* s,
                                                 double* t, double* ds, double* dt, const int* pair, const int* slot,
                                                 int a, int ipnof, const double* hpp, const double* J, const double* K,
                                                 double* parts, double* w, double tol, int maxit, double lr0,
                                                 double* info) {
    __shared__ double red[1024];
    __shared__ int hinit;
    const int tid = threadIdx.x, ng = npair * ncwo;
    double* xt = w;
    double* gc = w + ng;
    double* gt = w + 2 * ng;
    double* sv = w + 3 * ng;
    double* yv = w + 4 * ng;
    double* d = w + 5 * ng;
    double* Hinv = w + 6 * ng;
    if (tid == 0) hinit = 0;
    double E = on_eval_block(gamma, gc, npair, ncwo, isoftmax, s, t, ds, dt, pair, slot, a, ipnof, hpp, J, K,
                             parts, red);
    int it = 0;
    double gmax = 0.0;
    while (true) {
        double m = 0.0;
        for (int k = tid; k < ng; k += blockDim.x) m = fmax(m, fabs(gc[k]));
        gmax = block_max(m, red);
        if (!(gmax >= tol) || it >= maxit) break;  // also stops on a NaN gradient
        // direction: -lr0 g before the first curvature pair, else -H g
        const int hi = hinit;
        for (int k = tid; k < ng; k += blockDim.x) {
            double v;
            if (!hi) {
                v = -lr0 * gc[k];
            } else {
                v = 0.0;
                for (int j = 0; j < ng; ++j) v -= Hinv[(long long)k * ng + j] * gc[j];
            }
            d[k] = v;
        }
        __syncthreads();
        double part = 0.0;
        for (int k = tid; k < ng; k += blockDim.x) part += d[k] * gc[k];
        double dg = block_sum(part, red);
        if (dg >= 0.0) {  // not a descent direction: restart from the gradient
            if (tid == 0) hinit = 0;
            for (int k = tid; k < ng; k += blockDim.x) d[k] = -lr0 * gc[k];
            __syncthreads();
            part = 0.0;
            for (int k = tid; k < ng; k += blockDim.x) part += d[k] * gc[k];
            dg = block_sum(part, red);
        }
        double alpha = 1.0, Et = 0.0;
        bool failed = false;
        while (true) {
            for (int k = tid; k < ng; k += blockDim.x) xt[k] = gamma[k] + alpha * d[k];
            __syncthreads();
            Et = on_eval_block(xt, gt, npair, ncwo, isoftmax, s, t, ds, dt, pair, slot, a, ipnof, hpp, J, K, parts,
                               red);
            if (Et <= E + 1e-4 * alpha * dg || alpha * fabs(dg) < 1e-13 * fmax(1.0, fabs(E))) break;
            alpha *= 0.5;
            if (alpha < 1e-12) {
                failed = true;
                break;
            }
        }
        if (failed) break;
        // curvature pair and the BFGS update of H
        double psy = 0.0, pyy = 0.0;
        for (int k = tid; k < ng; k += blockDim.x) {
            sv[k] = xt[k] - gamma[k];
            yv[k] = gt[k] - gc[k];
            psy += sv[k] * yv[k];
            pyy += yv[k] * yv[k];
        }
        const double sy = block_sum(psy, red), yy = block_sum(pyy, red);
        if (sy > 0.0) {
            if (!hinit) {
                for (long long i = tid; i < (long long)ng * ng; i += blockDim.x)
                    Hinv[i] = (i / ng == i % ng) ? sy / yy : 0.0;
                __syncthreads();
                if (tid == 0) hinit = 1;
            }
            const double rho = 1.0 / sy;
            // H y into d (the direction is no longer needed)
            for (int k = tid; k < ng; k += blockDim.x) {
                double v = 0.0;
                for (int j = 0; j < ng; ++j) v += Hinv[(long long)k * ng + j] * yv[j];
                d[k] = v;
            }
            __syncthreads();
            part = 0.0;
            for (int k = tid; k < ng; k += blockDim.x) part += yv[k] * d[k];
            const double yHy = block_sum(part, red);
            const double cs = rho * rho * yHy + rho;
            for (long long i = tid; i < (long long)ng * ng; i += blockDim.x) {
                const int k = (int)(i / ng), j = (int)(i % ng);
                Hinv[i] += -rho * (sv[k] * d[j] + d[k] * sv[j]) + cs * sv[k] * sv[j];
            }
        }
        for (int k = tid; k < ng; k += blockDim.x) {
            gamma[k] = xt[k];
            gc[k] = gt[k];
        }
        __syncthreads();
        E = Et;
        ++it;
    }
    if (tid == 0) {
        info[0] = (double)it;
        info[1] = gmax;
    }
}

__global__ void k_gamma_descent(double* gamma, const double* grad, double lr, int ng) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < ng) gamma[k] -= lr * grad[k];
}

// ADAM moments and rotation generator y = -lr mhat / (sqrt(vhat) + eps)
__global__ void k_adam(const double* g, double* m, double* v, double* y, long long nn, double b1,
                       double b2, double c1, double c2, double lr, double eps, const int* tdev) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nn) return;
    if (tdev) {  // bias corrections of step t = *tdev + 1 (the counter is advanced by k_tick)
        const int t = *tdev + 1;
        c1 = 1.0 - pow(b1, (double)t);
        c2 = 1.0 - pow(b2, (double)t);
    }
    double gi = g[i];
    double mi = b1 * m[i] + (1.0 - b1) * gi;
    double vi = b2 * v[i] + (1.0 - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    y[i] = -lr * (mi / c1) / (sqrt(vi / c2) + eps);
}

__global__ void k_tick(int* t) { *t += 1; }

// out[0] = E, out[1] = ||g||_F, out[2] = max |lambda - lambda^T|
__global__ void k_step_stats(const double* E, const double* g, const double* lam, int n, int a,
                             double* out) {
    __shared__ double r1[256], r2[256];
    double s = 0.0, mx = 0.0;
    for (long long i = threadIdx.x; i < (long long)n * n; i += blockDim.x) {
        s = fma(g[i], g[i], s);
        int p = (int)(i / n), q = (int)(i % n);
        const double lpq = q < a ? lam[i] : 0.0, lqp = p < a ? lam[(long long)q * n + p] : 0.0;
        mx = fmax(mx, fabs(lpq - lqp));
    }
    r1[threadIdx.x] = s;
    r2[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) {
            r1[threadIdx.x] += r1[threadIdx.x + o];
            r2[threadIdx.x] = fmax(r2[threadIdx.x], r2[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = *E;
        out[1] = sqrt(r1[0]);
        out[2] = r2[0];
    }
}

}  // namespace

// ---------------------------------------------------------------------------------------
int pnof_occupations(nof_ctx* c, const double* gamma, cudaStream_t st) {
    if (c->opt.isoftmax)
        k_occupations_softmax<<<nblk(c->npair, 128), 128, 0, st>>>(gamma, c->npair, c->opt.ncwo, c->s, c->t,
                                                                     c->ds, c->dt);
    else
        k_occupations<<<nblk(c->npair, 128), 128, 0, st>>>(gamma, c->npair, c->opt.ncwo, c->s, c->t, c->ds,
                                                             c->dt);
    NOF_LAUNCH_CHECK();
    long long aa = (long long)c->nact * c->nact;
    float2 *Adf = nullptr, *Bcdf = nullptr;
    fast_coefficient_buffers(c, &Adf, &Bcdf);
    k_coefficients<<<nblk(aa), 256, 0, st>>>(c->s, c->t, c->pair, c->slot, c->nact,
                                                    c->opt.ipnof, c->occ, c->A, c->Bc, Adf, Bcdf);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

int pnof_hpp(nof_ctx* c, const double* C, cudaStream_t st) {
    const int n = c->nbf, a = c->nact;
    Gemm64 g;  // HC = H C_a
    g.M = n; g.N = a; g.K = n;
    g.A = c->H; g.sAm = n; g.sAk0 = 1;
    g.B = C; g.sBn = 1; g.sBk0 = n;
    g.C = c->HC; g.sCm = a; g.sCn = 1;
    g.work = c->gwork; g.work_cap = c->gwork_cap;
    NOF_TRY(gemm64(g, st));
    k_hpp<<<nblk((long long)a * 32), 256, 0, st>>>(C, c->HC, n, a, c->hpp);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

// E (into c->E) and dE/dgamma (into out) from J, K, h_pp and the occupations of pnof_occupations.
int pnof_gamma_grad(nof_ctx* c, double* out, cudaStream_t st) {
    const int a = c->nact;
    k_dE_parts<<<nblk((long long)a * 32), 256, 0, st>>>(c->s, c->t, c->pair, c->slot, c->hpp,
                                                               c->J, c->K, c->A, c->Bc, a, c->opt.ipnof,
                                                               c->part);
    NOF_LAUNCH_CHECK();
    k_gamma_chain<<<nblk(c->ngamma, 128), 128, 0, st>>>(c->s, c->t, c->ds, c->dt, c->slot,
                                                                c->part, c->npair, c->opt.ncwo, a, c->vnn,
                                                                c->E, out, c->status);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

int pnof_energy(nof_ctx* c, cudaStream_t st) { return pnof_gamma_grad(c, c->ggam, st); }

int pnof_jk_from_b(nof_ctx* c) {
    const int X = c->naux, a = c->nact;
    k_diag<<<nblk((long long)X * a), 256, 0, c->stream>>>(c->b, X, a, c->d);
    NOF_LAUNCH_CHECK();
    Gemm64 g;  // J = d^T d
    g.M = a; g.N = a; g.K = X;
    g.A = c->d; g.sAm = 1; g.sAk0 = a;
    g.B = c->d; g.sBn = 1; g.sBk0 = a;
    g.C = c->J; g.sCm = a; g.sCn = 1;
    g.work = c->gwork; g.work_cap = c->gwork_cap;
    NOF_TRY(gemm64(g, c->stream));
    k_ksum<<<nblk((long long)a * a), 256, 0, c->stream>>>(c->b, X, a, c->K);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

int pnof_build_W(nof_ctx* c) {
    const int X = c->naux, a = c->nact;
    Gemm64 g;  // D[P][p] = sum_r d[P][r] A[p][r]
    g.M = X; g.N = a; g.K = a;
    g.A = c->d; g.sAm = a; g.sAk0 = 1;
    g.B = c->A; g.sBn = a; g.sBk0 = 1;
    g.C = c->D; g.sCm = a; g.sCn = 1;
    g.work = c->gwork; g.work_cap = c->gwork_cap;
    NOF_TRY(gemm64(g, c->stream));
    k_build_W<<<nblk((long long)X * a * a), 256, 0, c->stream>>>(c->b, c->D, c->Bc, X, a, c->W);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

// Lam holds sum_P T^P W^P (assembled = false) or already Lambda (assembled = true); finish
// Lambda, lambda = C^T Lambda (columns p < a) and g.
int pnof_lambda_and_g(nof_ctx* c, const double* C, double* g_out, bool assembled) {
    const int n = c->nbf, a = c->nact;
    if (!assembled) {
        k_lambda_assemble<<<nblk((long long)n * a), 256, 0, c->stream>>>(c->HC, c->occ, n, a, c->Lam);
        NOF_LAUNCH_CHECK();
    }
    Gemm64 g;  // lam[q][p] = sum_mu C[mu][q] Lam[mu][p], p < a
    g.M = n; g.N = a; g.K = n;
    g.A = C; g.sAm = 1; g.sAk0 = n;
    g.B = c->Lam; g.sBn = 1; g.sBk0 = a;
    g.C = c->lam; g.sCm = n; g.sCn = 1;
    g.work = c->gwork; g.work_cap = c->gwork_cap;
    if (const int splits = gemm64_small_splits(g)) {
        // split-K partials, then lambda and g from them in one kernel
        NOF_TRY(gemm64_small_partials(g, splits, c->stream));
        k_reduce_gradient<<<nblk((long long)n * n), 256, 0, c->stream>>>(c->gwork, splits, n, a, c->lam, g_out);
        NOF_LAUNCH_CHECK();
        return NOF_OK;
    }
    NOF_TRY(gemm64(g, c->stream));
    k_orbital_gradient<<<nblk((long long)n * n), 256, 0, c->stream>>>(c->lam, n, a, g_out);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

// Plain FP64 JK stage: T = B C_a, b^P = C_a^T T^P, d, J, K, HC and h_pp.
int plain_jk(nof_ctx* c, const double* C) {
    const int n = c->nbf, X = c->naux, a = c->nact;
    cudaStream_t st = c->stream;
    {   // T[P][mu][p] = sum_nu B[P][mu][nu] C[nu][p]
        Gemm64 g;
        g.M = X * n; g.N = a; g.K = n;
        g.A = c->B; g.sAm = n; g.sAk0 = 1;
        g.B = C; g.sBn = 1; g.sBk0 = n;
        g.C = c->T; g.sCm = a; g.sCn = 1;
        NOF_TRY(prof_begin(c, "k_gemm64 (half transform T = B C)"));
        NOF_TRY(gemm64(g, st));
        NOF_TRY(prof_end(c));
    }
    {   // b[P][q][p] = sum_mu C[mu][q] T[P][mu][p]
        Gemm64 g;
        g.M = a; g.N = a; g.K = n; g.batch = X;
        g.A = C; g.sAm = 1; g.sAk0 = n; g.bA = 0;
        g.B = c->T; g.sBn = 1; g.sBk0 = a; g.bB = (long long)n * a;
        g.C = c->b; g.sCm = a; g.sCn = 1; g.bC = (long long)a * a;
        NOF_TRY(gemm64(g, st));
    }
    NOF_TRY(pnof_jk_from_b(c));
    NOF_TRY(pnof_hpp(c, C));
    return NOF_OK;
}

// Plain FP64 energy/gradient stage after plain_jk: occupations, coefficients and E at gamma;
// with want_grad also Lambda, lambda, g (into c->gorb) and dE/dgamma (into c->ggam).
int plain_grad(nof_ctx* c, const double* C, const double* gamma, bool want_grad) {
    const int n = c->nbf, X = c->naux, a = c->nact;
    cudaStream_t st = c->stream;
    NOF_TRY(pnof_occupations(c, gamma));
    NOF_TRY(pnof_energy(c, c->stream));
    if (!want_grad) return NOF_OK;
    NOF_TRY(pnof_build_W(c));
    {   // Lam[mu][p] = sum_{P,r} T[P][mu][r] W[P][r][p]  (composite contraction index)
        Gemm64 g;
        g.M = n; g.N = a; g.K = X * a; g.K0 = a;
        g.A = c->T; g.sAm = a; g.sAk0 = 1; g.sAk1 = (long long)n * a;
        g.B = c->W; g.sBn = 1; g.sBk0 = a; g.sBk1 = (long long)a * a;
        g.C = c->Lam; g.sCm = a; g.sCn = 1;
        int tiles = ((n + 63) / 64) * ((a + 63) / 64);
        int splits = 304 / tiles;
        if (splits < 1) splits = 1;
        int maxs = (X * a + 63) / 64;
        if (splits > maxs) splits = maxs;
        if ((size_t)splits * n * a > c->part_elems) splits = (int)(c->part_elems / ((size_t)n * a));
        if (splits < 1) splits = 1;
        NOF_TRY(gemm64_splitk(g, splits, c->W + (long long)X * a * a, st));
    }
    return pnof_lambda_and_g(c, C, c->gorb, false);
}

// ON update of an alternating step (see nof.h): on_iters steepest-descent steps on gamma with
// J, K and h_pp of the current orbitals held fixed.
int pnof_on_update(nof_ctx* c, double* gamma) {
    cudaStream_t st = c->stream;
    if (c->nact <= 256) {  // one block does every iteration
        if (c->opt.on_iters <= 0) return NOF_OK;
        float2 *Adf = nullptr, *Bcdf = nullptr;
        fast_coefficient_buffers(c, &Adf, &Bcdf);
        k_on_update_fused<<<1, 1024, 0, st>>>(gamma, c->npair, c->opt.ncwo, c->opt.isoftmax, c->s, c->t, c->ds, c->dt,
                                               c->pair, c->slot, c->nact, c->opt.ipnof, c->occ, c->A, c->Bc, Adf,
                                               Bcdf, c->hpp, c->J, c->K, c->part, c->ggam, c->opt.on_lr,
                                               c->opt.on_iters);
        NOF_LAUNCH_CHECK();
        return NOF_OK;
    }
    for (int it = 0; it < c->opt.on_iters; ++it) {
        NOF_TRY(pnof_occupations(c, gamma));
        NOF_TRY(pnof_gamma_grad(c, c->ggam, c->stream));
        k_gamma_descent<<<nblk(c->ngamma, 128), 128, 0, st>>>(gamma, c->ggam, c->opt.on_lr, c->ngamma);
        NOF_LAUNCH_CHECK();
    }
    return NOF_OK;
}

// ADAM moments and the rotation generator y from gradient g at step t (host counter, t >= 1).
int pnof_adam_y(nof_ctx* c, const double* g, double* m, double* v, double* y, int t, double lr, double eps) {
    const long long nn = (long long)c->nbf * c->nbf;
    const double c1 = 1.0 - std::pow(c->opt.b1, t), c2 = 1.0 - std::pow(c->opt.b2, t);
    k_adam<<<nblk(nn), 256, 0, c->stream>>>(g, m, v, y, nn, c->opt.b1, c->opt.b2, c1, c2, lr, eps, nullptr);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

// out[0] = E, out[1] = ||g||_F, out[2] = max |lambda - lambda^T| of the context's last evaluation.
int pnof_step_stats(nof_ctx* c, const double* g, double* out) {
    k_step_stats<<<1, 256, 0, c->stream>>>(c->E, g, c->lam, c->nbf, c->nact, out);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

// ONs converged at the J, K and h_pp of the context's last transform (see k_on_bfgs); w: 6 ng + ng^2
// doubles of scratch, info: 2 device doubles.
int pnof_on_converge(nof_ctx* c, double* gamma, double tol, int maxit, double lr0, double* w, double* info) {
    k_on_bfgs<<<1, 1024, 0, c->stream>>>(gamma, c->npair, c->opt.ncwo, c->opt.isoftmax, c->s, c->t, c->ds, c->dt,
                                         c->pair, c->slot, c->nact, c->opt.ipnof, c->hpp, c->J, c->K, c->part, w, tol,
                                         maxit, lr0, info);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

// ADAM update, rotation and statistics (called after the gradient at gamma_new is ready).
int pnof_adam_rotate(nof_ctx* c, double* C, double* m, double* v, int* t, double* out) {
    const int n = c->nbf;
    cudaStream_t st = c->stream;
    long long nn = (long long)n * n;
    double c1 = 0.0, c2 = 0.0;
    if (t) {
        *t += 1;
        c1 = 1.0 - std::pow(c->opt.b1, *t);
        c2 = 1.0 - std::pow(c->opt.b2, *t);
    }
    k_adam<<<nblk(nn), 256, 0, st>>>(c->gorb, m, v, c->y, nn, c->opt.b1, c->opt.b2, c1, c2,
                                     c->opt.lr, c->opt.eps, t ? nullptr : c->tdev);
    NOF_LAUNCH_CHECK();
    if (!t) {
        k_tick<<<1, 1, 0, st>>>(c->tdev);
        NOF_LAUNCH_CHECK();
    }
    k_step_stats<<<1, 256, 0, st>>>(c->E, c->gorb, c->lam, n, c->nact, out);
    NOF_LAUNCH_CHECK();
    if (t)
        NOF_TRY(expm_antisym_device(c->y, c->U, c->U2, c->tmpn, n, st, c->gwork, c->gwork_cap));
    else
        NOF_TRY(expm_antisym_device_fixed(c->y, c->U, c->U2, c->tmpn, n, c->status, st, c->gwork,
                                          c->gwork_cap));
    Gemm64 g;  // tmp = C U
    g.M = n; g.N = n; g.K = n;
    g.A = C; g.sAm = n; g.sAk0 = 1;
    g.B = c->U; g.sBn = 1; g.sBk0 = n;
    g.C = c->tmpn; g.sCm = n; g.sCn = 1;
    g.work = c->gwork; g.work_cap = c->gwork_cap;
    NOF_TRY(gemm64(g, st));
    NOF_CUDA(cudaMemcpyAsync(C, c->tmpn, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return NOF_OK;
}
