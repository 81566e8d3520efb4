// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/nof.h"

// ---------------------------------------------------------------------------------------
// Error handling: every entry point returns an int status; the message is thread-local.
// ---------------------------------------------------------------------------------------
void nof_set_error(const std::string& msg);
int nof_cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define NOF_CUDA(call)                                                            \
    do {                                                                          \
        cudaError_t e__ = (call);                                                 \
        if (e__ != cudaSuccess) return nof_cuda_fail(e__, #call, __FILE__, __LINE__); \
    } while (0)
// Every kernel launch site is followed by NOF_LAUNCH_CHECK, which also counts the launch.
void nof_count_launch();
#define NOF_LAUNCH_CHECK()       \
    do {                         \
        nof_count_launch();      \
        NOF_CUDA(cudaGetLastError()); \
    } while (0)
#define NOF_TRY(expr)              \
    do {                           \
        int r__ = (expr);          \
        if (r__ != NOF_OK) return r__; \
    } while (0)

// Device status word bits (written by kernels, read by nof_sync).
enum { NOF_DEV_NONFINITE = 1, NOF_DEV_TIMEOUT = 2, NOF_DEV_ILLCOND = 4, NOF_DEV_RANGE = 8 };

// ---------------------------------------------------------------------------------------
// Split-precision (exact BF16 digit) storage of the RI tensor; defined in fast.cu.
// ---------------------------------------------------------------------------------------
struct FastState;

struct nof_ctx {
    nof_options opt;
    cudaStream_t stream;
    int built;
    int natom, nbf, naux, nact, ngamma, nelec, npair;
    // basis description on the device
    int *fn_atom, *fn_first, *fn_nprim;   // per orbital function
    double *pexp, *pcoef;                  // orbital primitives (coef normalised in place)
    int *ax_atom;                          // per aux function
    double *axexp;
    double *xyz, *Z;
    // one-electron and RI data
    double *S, *H, *vnn;
    double *B;        // FP64 [X][n][n] (plain path; also the source of the digit planes)
    // pairing structure
    int *pair, *slot;
    // workspaces for an evaluation (plain path)
    double *T, *b, *d, *J, *K, *D, *W, *HC, *Lam, *lam, *hpp, *A, *Bc;
    double *s, *t, *ds, *dt, *occ, *E, *part, *ggam, *gorb;
    size_t part_elems;
    // step workspaces
    double *y, *U, *U2, *tmpn;
    double* gwork;  // split-K scratch of the FP64 GEMMs
    size_t gwork_cap;
    int* status;
    FastState* fast;
    // fork/join events of the batched evaluation
    cudaEvent_t ev_fork, ev_join;
    // low-priority side stream of a split-precision evaluation (the work off the gradient's
    // chain) and its events: fork, occupations written, T written, b written, the rest of the
    // gradient's side inputs written, J/K and energy done
    cudaStream_t side;
    cudaEvent_t ev_s0, ev_sO, ev_sT, ev_sJ, ev_s1, ev_s2;
    // recorded graphs of nof_energy_grad (option graphs), the least recently used replaced first:
    // the argument pointers each was recorded with and the kernel launches it holds; the pointer
    // sets of recent direct calls (a set is recorded on its second call); a flag set when
    // recording failed once (the context then launches directly)
    struct EvalGraph {
        cudaGraphExec_t exec;
        const void* key[5];
        long long kernels;
        unsigned long long used;
    };
    static constexpr int kEvalGraphs = 4;
    EvalGraph geval[kEvalGraphs];
    const void* gseen[kEvalGraphs][5];
    int gseen_next;
    unsigned long long gtick;
    int gfail;
    // static field (nof_set_field): dipole integrals [3][n][n], the field-free h and V_nn,
    // scratch of the dipole moment [3][a]; all allocated on first use
    double *Dip, *H0, *vnn0, *dipw;
    // ADAM step counter on the device for nof_step with t == NULL (zero after nof_build_B)
    int* tdev;
    // converged loop (nof_optimize): one allocation made on its first call, freed by nof_destroy
    double* opt_buf;
    size_t opt_cap;
    // nuclear gradient (FP64 path): L^-1 of the Coulomb metric kept from set-up, and workspaces
    // allocated on the first nof_nuclear_gradient
    double *Linv, *gr_cfit, *gr_Y, *gr_Gam, *gr_Z, *gr_small;
    // timing of one contraction (nof_profile): 0 off, 1..3 the contraction bracketed
    int prof_on;
    const char* prof_name;
    void* prof_events;  // std::vector<std::pair<cudaEvent_t, cudaEvent_t>>*
};

// Bracket one contraction of an evaluation with timing events when profiling selects it
// (which: 1 half transform, 2 full transform, 3 Lagrangian contraction; nof_profile).
int prof_begin(nof_ctx* c, const char* name, int which = 1);
int prof_end(nof_ctx* c, int which = 1);

// ---------------------------------------------------------------------------------------
// FP64 building blocks (linalg.cu)
// ---------------------------------------------------------------------------------------
// Generic strided FP64 GEMM: C(m,n) = alpha * sum_k A(m,k) B(k,n) + beta * C(m,n).
// The contraction index may be two-level: k = k1 * K0 + k0 with element offsets
// k0 * s?k0 + k1 * s?k1 (lets one GEMM run over a composite (P, r) index).
// Batched over grid z with element strides bA, bB, bC.
struct Gemm64 {
    int M = 0, N = 0, K = 0, K0 = 1 << 30, batch = 1;
    const double* A = nullptr;
    long long sAm = 0, sAk0 = 0, sAk1 = 0, bA = 0;
    const double* B = nullptr;
    long long sBn = 0, sBk0 = 0, sBk1 = 0, bB = 0;
    double* C = nullptr;
    long long sCm = 0, sCn = 1, bC = 0;
    double alpha = 1.0, beta = 0.0;
    bool a_lower = false;  // A(m, k) = 0 for k > m: each output row block stops its K loop there
    // Optional scratch for an automatic split-K when the output has too few 64x64 tiles to fill
    // the GPU (FP64 runs at 2 FMA/clk/SM on GB300, so a single CTA per tile is far too slow).
    double* work = nullptr;
    size_t work_cap = 0;  // doubles
};
int gemm64(const Gemm64& g, cudaStream_t st);
// Same contraction with the K range split over `splits` CTAs; partial results are written
// to work[split][M][N] then summed in a fixed order into C (deterministic).
int gemm64_splitk(const Gemm64& g, int splits, double* work, cudaStream_t st);
// The small-output route of gemm64 in two steps: the K split it takes (0 when it does not take
// that route), and the launch that writes the split's partial products to g.work[split][M][N]
// (summed afterwards in split order, like gemm64 does).
int gemm64_small_splits(const Gemm64& g);
int gemm64_small_partials(const Gemm64& g, int splits, cudaStream_t st);

int cholesky_inverse(double* V, double* Linv, int X, int* status, cudaStream_t st);
int newton_schulz_invsqrt(const double* S, double* Xout, double* w1, double* w2, double* w3,
                          double* w4, int n, int iters, cudaStream_t st, double* work = nullptr,
                          size_t work_cap = 0);
int expm_antisym_device(const double* y, double* U, double* w1, double* w2, int n,
                        cudaStream_t st, double* work = nullptr, size_t work_cap = 0);
// The same series with a fixed scaling 2^-12 and 12 squarings: no host synchronisation, so it can
// be captured in a CUDA graph. Sets NOF_DEV_RANGE in *status when ||y||_F > 2^12 (the scaled
// norm would exceed 1).
int expm_antisym_device_fixed(const double* y, double* U, double* w1, double* w2, int n, int* status,
                              cudaStream_t st, double* work = nullptr, size_t work_cap = 0);

int sym_eig(double* A, double* Vwork, double* Vout, double* w, int n, int* sweeps_dev, cudaStream_t st);

// Integrals (integrals.cu)
int build_integrals(nof_ctx* c, double* M3 /* [X][n][n] */, double* V2 /* [X][X] */);

// PNOF kernels (pnof.cu)
int plain_jk(nof_ctx* c, const double* C);
int plain_grad(nof_ctx* c, const double* C, const double* gamma, bool want_grad);
int pnof_occupations(nof_ctx* c, const double* gamma, cudaStream_t st);
inline int pnof_occupations(nof_ctx* c, const double* gamma) { return pnof_occupations(c, gamma, c->stream); }
int pnof_energy(nof_ctx* c, cudaStream_t st);
int pnof_gamma_grad(nof_ctx* c, double* out, cudaStream_t st);
int pnof_hpp(nof_ctx* c, const double* C, cudaStream_t st);
inline int pnof_hpp(nof_ctx* c, const double* C) { return pnof_hpp(c, C, c->stream); }
int pnof_lambda_and_g(nof_ctx* c, const double* C, double* g_out, bool assembled);
int pnof_jk_from_b(nof_ctx* c);
int pnof_build_W(nof_ctx* c);
int pnof_on_update(nof_ctx* c, double* gamma);
int pnof_on_converge(nof_ctx* c, double* gamma, double tol, int maxit, double lr0, double* w, double* info);
int pnof_adam_y(nof_ctx* c, const double* g, double* m, double* v, double* y, int t, double lr, double eps);
int pnof_step_stats(nof_ctx* c, const double* g, double* out);
int pnof_adam_rotate(nof_ctx* c, double* C, double* m, double* v, int* t, double* out);

// Split-precision path (fast.cu)
int fast_prepare(nof_ctx* c);
int fast_release(nof_ctx* c);
int fast_jk(nof_ctx* c, const double* C);
int fast_grad(nof_ctx* c, const double* C, const double* gamma, bool want_grad);
int fast_eval(nof_ctx* c, const double* C, const double* gamma, bool want_grad);
int fast_get_B(nof_ctx* c, double* B);
int fast_tiles(nof_ctx* c, int* out);
int fast_digits(nof_ctx* c);
// split path: double-float copies of A and B for k_coefficients (null outside the split path)
void fast_coefficient_buffers(nof_ctx* c, float2** Adf, float2** Bcdf);
