// One- and two-electron integrals over s Gaussians on the device (FP64).
//
// The paper defines h_ki (kinetic energy plus nuclear attraction) and the Coulomb integrals
// <kl|ij> in its Theory section and evaluates them with libcint; for s functions they have
// closed forms. With p = a + b, P = (aA + bB)/p, K_AB = exp(-ab/p |A-B|^2):
//   S = (pi/p)^{3/2} K_AB,  T = (ab/p)(3 - 2(ab/p)|A-B|^2) S,
//   V = -Z_C (2pi/p) K_AB F0(p|P-C|^2),
//   (ab|cd) = 2 pi^{5/2} / (pq sqrt(p+q)) K_AB K_CD F0(pq/(p+q) |P-Q|^2),
// F0(t) = (1/2) sqrt(pi/t) erf(sqrt t), F0(0) = 1. The RI three-centre (P|mu nu) and the
// Coulomb metric (P|Q) are the repulsion formula with single-Gaussian aux functions.
#include <cmath>

#include "internal.h"

namespace {

__device__ __forceinline__ double boys0(double t) {
    if (t < 1e-8) return 1.0 - t / 3.0 + t * t / 10.0;
    double st = sqrt(t);
    return 0.88622692545275801365 * erf(st) / st;  // sqrt(pi)/2 * erf(sqrt t)/sqrt t
}

__device__ __forceinline__ double prim_norm(double a) {
    return pow(2.0 * a / 3.14159265358979323846, 0.75);
}

// Normalise every contracted orbital function in place: primitive norms, then the contraction.
__global__ void k_norm_orb(const int* fn_first, const int* fn_nprim, const double* pexp,
                           double* pcoef, int n) {
    int mu = blockIdx.x * blockDim.x + threadIdx.x;
    if (mu >= n) return;
    int f = fn_first[mu], np = fn_nprim[mu];
    for (int i = 0; i < np; ++i) pcoef[f + i] *= prim_norm(pexp[f + i]);
    double s = 0.0;
    for (int i = 0; i < np; ++i)
        for (int j = 0; j < np; ++j) {
            double p = pexp[f + i] + pexp[f + j];
            s += pcoef[f + i] * pcoef[f + j] * pow(3.14159265358979323846 / p, 1.5);
        }
    double r = 1.0 / sqrt(s);
    for (int i = 0; i < np; ++i) pcoef[f + i] *= r;
}

__global__ void k_one_electron(const int* fn_atom, const int* fn_first, const int* fn_nprim,
                               const double* pexp, const double* pcoef, const double* xyz,
                               const double* Z, int natom, int n, double* S, double* H) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    int mu = (int)(idx / n), nu = (int)(idx % n);
    const double* A = xyz + 3 * fn_atom[mu];
    const double* Bc = xyz + 3 * fn_atom[nu];
    double ab2 = (A[0] - Bc[0]) * (A[0] - Bc[0]) + (A[1] - Bc[1]) * (A[1] - Bc[1]) +
                 (A[2] - Bc[2]) * (A[2] - Bc[2]);
    double s = 0.0, t = 0.0, v = 0.0;
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < fn_nprim[mu]; ++i) {
        double a = pexp[fn_first[mu] + i], ca = pcoef[fn_first[mu] + i];
        for (int j = 0; j < fn_nprim[nu]; ++j) {
            double b = pexp[fn_first[nu] + j], cb = pcoef[fn_first[nu] + j];
            double p = a + b, red = a * b / p;
            double K = exp(-red * ab2);
            double sp = pow(pi / p, 1.5) * K;
            s += ca * cb * sp;
            t += ca * cb * red * (3.0 - 2.0 * red * ab2) * sp;
            double P0 = (a * A[0] + b * Bc[0]) / p, P1 = (a * A[1] + b * Bc[1]) / p,
                   P2 = (a * A[2] + b * Bc[2]) / p;
            double vs = 0.0;
            for (int c = 0; c < natom; ++c) {
                const double* Cc = xyz + 3 * c;
                double pc2 = (P0 - Cc[0]) * (P0 - Cc[0]) + (P1 - Cc[1]) * (P1 - Cc[1]) +
                             (P2 - Cc[2]) * (P2 - Cc[2]);
                vs -= Z[c] * boys0(p * pc2);
            }
            v += ca * cb * (2.0 * pi / p) * K * vs;
        }
    }
    S[idx] = s;
    H[idx] = t + v;
}

__global__ void k_two_center(const int* ax_atom, const double* axexp, const double* xyz, int X,
                             double* V) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)X * X) return;
    int P = (int)(idx / X), Q = (int)(idx % X);
    const double* A = xyz + 3 * ax_atom[P];
    const double* Bc = xyz + 3 * ax_atom[Q];
    double r2 = (A[0] - Bc[0]) * (A[0] - Bc[0]) + (A[1] - Bc[1]) * (A[1] - Bc[1]) +
                (A[2] - Bc[2]) * (A[2] - Bc[2]);
    double p = axexp[P], q = axexp[Q];
    const double pi = 3.14159265358979323846;
    V[idx] = prim_norm(p) * prim_norm(q) * 2.0 * pow(pi, 2.5) / (p * q * sqrt(p + q)) *
             boys0(p * q / (p + q) * r2);
}

// (P|mu nu) for mu <= nu, packed row-major upper triangle: column index
// mu*n - mu(mu-1)/2 + (nu - mu).
__global__ void k_three_center(const int* fn_atom, const int* fn_first, const int* fn_nprim,
                               const double* pexp, const double* pcoef, const int* ax_atom,
                               const double* axexp, const double* xyz, int n, int X,
                               double* M) {
    long long npk = (long long)n * (n + 1) / 2;
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= npk * X) return;
    int P = (int)(idx / npk);
    long long c = idx - P * npk;
    // invert the packed index: largest mu with start(mu) <= c
    int mu = (int)((2.0 * n + 1 - sqrt((2.0 * n + 1) * (2.0 * n + 1) - 8.0 * (double)c)) / 2.0);
    if (mu < 0) mu = 0;
    while (mu > 0 && (long long)mu * n - (long long)mu * (mu - 1) / 2 > c) --mu;
    while ((long long)(mu + 1) * n - (long long)(mu + 1) * mu / 2 <= c) ++mu;
    int nu = mu + (int)(c - ((long long)mu * n - (long long)mu * (mu - 1) / 2));
    const double* A = xyz + 3 * fn_atom[mu];
    const double* Bc = xyz + 3 * fn_atom[nu];
    const double* Cc = xyz + 3 * ax_atom[P];
    double q = axexp[P];
    double ab2 = (A[0] - Bc[0]) * (A[0] - Bc[0]) + (A[1] - Bc[1]) * (A[1] - Bc[1]) +
                 (A[2] - Bc[2]) * (A[2] - Bc[2]);
    const double pi = 3.14159265358979323846;
    double acc = 0.0;
    for (int i = 0; i < fn_nprim[mu]; ++i) {
        double a = pexp[fn_first[mu] + i], ca = pcoef[fn_first[mu] + i];
        for (int j = 0; j < fn_nprim[nu]; ++j) {
            double b = pexp[fn_first[nu] + j], cb = pcoef[fn_first[nu] + j];
            double p = a + b;
            double K = exp(-a * b / p * ab2);
            double P0 = (a * A[0] + b * Bc[0]) / p - Cc[0], P1 = (a * A[1] + b * Bc[1]) / p - Cc[1],
                   P2 = (a * A[2] + b * Bc[2]) / p - Cc[2];
            double r2 = P0 * P0 + P1 * P1 + P2 * P2;
            acc += ca * cb * K * 2.0 * pow(pi, 2.5) / (p * q * sqrt(p + q)) *
                   boys0(p * q / (p + q) * r2);
        }
    }
    M[idx] = prim_norm(q) * acc;
}

__global__ void k_nuclear_repulsion(const double* xyz, const double* Z, int natom, double* out) {
    __shared__ double red[256];
    double s = 0.0;
    for (long long k = threadIdx.x; k < (long long)natom * natom; k += blockDim.x) {
        int A = (int)(k / natom), B = (int)(k % natom);
        if (B <= A) continue;
        double dx = xyz[3 * A] - xyz[3 * B], dy = xyz[3 * A + 1] - xyz[3 * B + 1],
               dz = xyz[3 * A + 2] - xyz[3 * B + 2];
        s += Z[A] * Z[B] / sqrt(dx * dx + dy * dy + dz * dz);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

inline unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// Fills S, H, vnn in the context and the packed (P|mu nu) and (P|Q) buffers.
int build_integrals(nof_ctx* c, double* M3, double* V2) {
    const int n = c->nbf, X = c->naux;
    cudaStream_t st = c->stream;
    k_norm_orb<<<nblk(n, 128), 128, 0, st>>>(c->fn_first, c->fn_nprim, c->pexp, c->pcoef, n);
    NOF_LAUNCH_CHECK();
    k_one_electron<<<nblk((long long)n * n), 256, 0, st>>>(c->fn_atom, c->fn_first, c->fn_nprim,
                                                           c->pexp, c->pcoef, c->xyz, c->Z,
                                                           c->natom, n, c->S, c->H);
    NOF_LAUNCH_CHECK();
    k_nuclear_repulsion<<<1, 256, 0, st>>>(c->xyz, c->Z, c->natom, c->vnn);
    NOF_LAUNCH_CHECK();
    k_two_center<<<nblk((long long)X * X), 256, 0, st>>>(c->ax_atom, c->axexp, c->xyz, X, V2);
    NOF_LAUNCH_CHECK();
    long long npk = (long long)n * (n + 1) / 2;
    k_three_center<<<nblk(npk * X), 256, 0, st>>>(c->fn_atom, c->fn_first, c->fn_nprim, c->pexp,
                                                  c->pcoef, c->ax_atom, c->axexp, c->xyz, n, X, M3);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}
