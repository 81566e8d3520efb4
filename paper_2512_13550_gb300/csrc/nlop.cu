// Finite-field workload (NLOPs subsection): the static field term of the Hamiltonian, the
// dipole moment of a state, the centred differences and the Romberg-Richardson triangle, and
// a batched step over independent field instances. C ABI in include/nof.h.
#include <cmath>
#include <limits>

#include "internal.h"

namespace {

inline unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// D[k][mu][nu] = <mu|r_k|nu> for contracted s functions: per primitive pair the product
// Gaussian sits at P = (a A + b B) / (a + b), so <a|r_k|b> = P_k <a|b>.
__global__ void k_dipole_integrals(const int* fn_atom, const int* fn_first, const int* fn_nprim,
                                   const double* pexp, const double* pcoef, const double* xyz, int n,
                                   double* D) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nn = (long long)n * n;
    if (idx >= nn) return;
    const int mu = (int)(idx / n), nu = (int)(idx % n);
    const double* A = xyz + 3 * fn_atom[mu];
    const double* B = xyz + 3 * fn_atom[nu];
    const double ab2 = (A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) + (A[2] - B[2]) * (A[2] - B[2]);
    const double pi = 3.14159265358979323846;
    double d0 = 0.0, d1 = 0.0, d2 = 0.0;
    for (int i = 0; i < fn_nprim[mu]; ++i) {
        const double a = pexp[fn_first[mu] + i], ca = pcoef[fn_first[mu] + i];
        for (int j = 0; j < fn_nprim[nu]; ++j) {
            const double b = pexp[fn_first[nu] + j], cb = pcoef[fn_first[nu] + j];
            const double p = a + b;
            const double w = ca * cb * pow(pi / p, 1.5) * exp(-a * b / p * ab2);
            d0 += w * (a * A[0] + b * B[0]) / p;
            d1 += w * (a * A[1] + b * B[1]) / p;
            d2 += w * (a * A[2] + b * B[2]) / p;
        }
    }
    D[idx] = d0;
    D[nn + idx] = d1;
    D[2 * nn + idx] = d2;
}

// h = h0 + F . D and (thread 0) V_nn = V_nn0 - F . sum_A Z_A R_A.
__global__ void k_field_h(const double* H0, const double* D, long long nn, double f0, double f1, double f2,
                          const double* vnn0, const double* xyz, const double* Z, int natom, double* H,
                          double* vnn) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx < nn) H[idx] = H0[idx] + f0 * D[idx] + f1 * D[nn + idx] + f2 * D[2 * nn + idx];
    if (idx == 0) {
        double m0 = 0.0, m1 = 0.0, m2 = 0.0;
        for (int A = 0; A < natom; ++A) {
            m0 += Z[A] * xyz[3 * A];
            m1 += Z[A] * xyz[3 * A + 1];
            m2 += Z[A] * xyz[3 * A + 2];
        }
        *vnn = *vnn0 - (f0 * m0 + f1 * m1 + f2 * m2);
    }
}

// w[k][p] = (C^T D_k C)_pp, one block per (p, k): a fixed-order tree sum over mu of
// C_mu,p sum_nu D_k,mu,nu C_nu,p.
__global__ void __launch_bounds__(256) k_dipole_diag(const double* C, const double* D, int n, int a, double* w) {
    __shared__ double red[256];
    const int p = blockIdx.x, k = blockIdx.y;
    const double* Dk = D + (long long)k * n * n;
    double acc = 0.0;
    for (int mu = threadIdx.x; mu < n; mu += 256) {
        double s = 0.0;
        for (int nu = 0; nu < n; ++nu) s += Dk[(long long)mu * n + nu] * C[(long long)nu * n + p];
        acc += C[(long long)mu * n + p] * s;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) w[k * a + p] = red[0];
}

// mu_k = -2 sum_p n_p w[k][p] + sum_A Z_A R_A,k: warp k, lane-strided sum then a shuffle tree.
__global__ void k_dipole_sum(const double* w, const double* occ, int a, const double* xyz, const double* Z,
                             int natom, double* mu) {
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= 3) return;
    double s = 0.0;
    for (int p = lane; p < a; p += 32) s += occ[p] * w[k * a + p];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        double nuc = 0.0;
        for (int A = 0; A < natom; ++A) nuc += Z[A] * xyz[3 * A + k];
        mu[k] = -2.0 * s + nuc;
    }
}

template <class T>
int alloc(T** p, size_t count) {
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return nof_cuda_fail(e, "cudaMalloc (field workspaces)", __FILE__, __LINE__);
    }
    return NOF_OK;
}

int check(nof_ctx* c) {
    if (!c) {
        nof_set_error("null context");
        return NOF_EINVAL;
    }
    if (!c->built) {
        nof_set_error("nof_build_B has not been called on this context");
        return NOF_ESTATE;
    }
    return NOF_OK;
}

// Dipole integrals and the field-free copies, on first use.
int ensure_field_state(nof_ctx* c) {
    const long long nn = (long long)c->nbf * c->nbf;
    if (!c->Dip) {
        NOF_TRY(alloc(&c->Dip, 3 * nn));
        k_dipole_integrals<<<blocks(nn), 256, 0, c->stream>>>(c->fn_atom, c->fn_first, c->fn_nprim, c->pexp,
                                                               c->pcoef, c->xyz, c->nbf, c->Dip);
        NOF_LAUNCH_CHECK();
    }
    if (!c->H0) {
        NOF_TRY(alloc(&c->H0, nn));
        NOF_TRY(alloc(&c->vnn0, 1));
        NOF_CUDA(cudaMemcpyAsync(c->H0, c->H, nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        NOF_CUDA(cudaMemcpyAsync(c->vnn0, c->vnn, sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    }
    if (!c->dipw) NOF_TRY(alloc(&c->dipw, 3 * (size_t)c->nact));
    return NOF_OK;
}

}  // namespace

extern "C" {

int nof_set_field(nof_ctx* c, const double* F) {
    NOF_TRY(check(c));
    if (!F || !std::isfinite(F[0]) || !std::isfinite(F[1]) || !std::isfinite(F[2])) {
        nof_set_error("nof_set_field: null or non-finite field");
        return NOF_EINVAL;
    }
    NOF_TRY(ensure_field_state(c));
    const long long nn = (long long)c->nbf * c->nbf;
    k_field_h<<<blocks(nn), 256, 0, c->stream>>>(c->H0, c->Dip, nn, F[0], F[1], F[2], c->vnn0, c->xyz, c->Z,
                                                  c->natom, c->H, c->vnn);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

int nof_dipole(nof_ctx* c, const double* C, const double* gamma, double* mu) {
    NOF_TRY(check(c));
    if (!C || !gamma || !mu) {
        nof_set_error("nof_dipole: null pointer");
        return NOF_EINVAL;
    }
    NOF_TRY(ensure_field_state(c));
    NOF_TRY(pnof_occupations(c, gamma));  // n_p into c->occ
    k_dipole_diag<<<dim3(c->nact, 3), 256, 0, c->stream>>>(C, c->Dip, c->nbf, c->nact, c->dipw);
    NOF_LAUNCH_CHECK();
    k_dipole_sum<<<1, 96, 0, c->stream>>>(c->dipw, c->occ, c->nact, c->xyz, c->Z, c->natom, mu);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

int nof_field_differences(const double* mu, int npoint, double step, double* alpha, double* beta,
                          double* gamma) {
    if (!mu || !alpha || !beta || !gamma || npoint < 1 || !(step > 0.0)) {
        nof_set_error("nof_field_differences: null pointer, npoint < 1 or step <= 0");
        return NOF_EINVAL;
    }
    const int L = npoint + 1;  // +h_1 .. +h_L at mu[1 .. L], -h_1 .. -h_L at mu[L + 1 .. 2L]
    const double m0 = mu[0];
    for (int k = 0; k < npoint; ++k) {
        const double h = std::ldexp(step, k);
        const double p1 = mu[1 + k], p2 = mu[2 + k], m1 = mu[L + 1 + k], m2 = mu[L + 2 + k];
        alpha[k] = (p1 - m1) / (2.0 * h);
        beta[k] = (p1 - 2.0 * m0 + m1) / (h * h);
        gamma[k] = (p2 - 2.0 * p1 + 2.0 * m1 - m2) / (2.0 * h * h * h);
    }
    return NOF_OK;
}

int nof_romberg(const double* D, int npoint, double* R, double* best, int* sel) {
    if (!D || !R || !best || !sel || npoint < 1) {
        nof_set_error("nof_romberg: null pointer or npoint < 1");
        return NOF_EINVAL;
    }
    const int N = npoint;
    const double nan = std::numeric_limits<double>::quiet_NaN();
    for (int i = 0; i < N * N; ++i) R[i] = nan;
    for (int k = 0; k < N; ++k) R[k * N] = D[k];
    for (int j = 2; j <= N; ++j)
        for (int k = 1; k <= N - j + 1; ++k) {
            const double prev = R[(k - 1) * N + j - 2], next = R[k * N + j - 2];
            R[(k - 1) * N + j - 1] = prev + (prev - next) / (std::ldexp(1.0, 2 * (j - 1)) - 1.0);
        }
    best[0] = D[0];
    best[1] = nan;
    sel[0] = sel[1] = 1;
    bool found = false;
    for (int j = 1; j < N; ++j)
        for (int k = 1; k <= N - j; ++k) {
            const double delta = std::fabs(R[k * N + j - 1] - R[(k - 1) * N + j - 1]);
            const double value = R[(k - 1) * N + j];
            if (!found || delta < best[1] || (delta == best[1] && std::fabs(value) < std::fabs(best[0]))) {
                best[0] = value;
                best[1] = delta;
                sel[0] = k;
                sel[1] = j;
                found = true;
            }
        }
    return NOF_OK;
}

int nof_polarizability_invariants(const double* a, double* out) {
    if (!a || !out) {
        nof_set_error("nof_polarizability_invariants: null pointer");
        return NOF_EINVAL;
    }
    out[0] = (a[0] + a[1] + a[2]) / 3.0;
    const double d01 = a[0] - a[1], d12 = a[1] - a[2], d20 = a[2] - a[0];
    out[1] = std::sqrt((d01 * d01 + d12 * d12 + d20 * d20) / 2.0);
    return NOF_OK;
}

int nof_step_batch(nof_ctx* const* ctxs, int count, double* const* C, double* const* gamma, double* const* m,
                   double* const* v, int* const* t, double* const* out, void* stream) {
    if (count <= 0 || !ctxs || !C || !gamma || !m || !v || !out) {
        nof_set_error("nof_step_batch: bad count or null array");
        return NOF_EINVAL;
    }
    for (int i = 0; i < count; ++i) {
        NOF_TRY(check(ctxs[i]));
        if (!C[i] || !gamma[i] || !m[i] || !v[i] || !out[i]) {
            nof_set_error("nof_step_batch: null entry");
            return NOF_EINVAL;
        }
    }
    cudaStream_t master = (cudaStream_t)stream;
    NOF_CUDA(cudaEventRecord(ctxs[0]->ev_fork, master));
    for (int i = 0; i < count; ++i) {
        nof_ctx* c = ctxs[i];
        NOF_CUDA(cudaStreamWaitEvent(c->stream, ctxs[0]->ev_fork, 0));
        NOF_TRY(nof_step(c, C[i], gamma[i], m[i], v[i], t ? t[i] : nullptr, out[i]));
        NOF_CUDA(cudaEventRecord(c->ev_join, c->stream));
        NOF_CUDA(cudaStreamWaitEvent(master, c->ev_join, 0));
    }
    return NOF_OK;
}

}  // extern "C"
