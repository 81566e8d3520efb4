// nof_jk_static: J and K from a caller-owned RI tensor and orbitals, with no device allocation.
//
// Some callers cannot call cudaMalloc: an application whose device memory is owned by another
// allocator (a framework's caching pool that has reserved the GPU, or a memory budget enforced
// by the host program), or code that must not stall or fail on an allocation in the middle of
// its run. For them this entry point keeps its scratch (the half-transformed tensor T, the fully
// transformed b, the diagonal d and the split-K partials of J) in one file-scope device array of
// fixed size, so a call only launches kernels on the caller's stream.
//
// When the array is reserved: this translation unit is its own CUDA module, and CUDA loads
// modules lazily by default (CUDA_MODULE_LOADING=LAZY), so the 48 MiB are reserved on a device
// when the module first loads there, which is inside the first nof_jk_static call made with that
// device current (the address look-up below loads it). With eager loading they are reserved when
// the library is loaded. Either way they stay reserved until the process exits. A caller that
// hands the GPU to a pool or a budget afterwards should make one call first, before doing so.
// The device address is looked up on that first call too; make it before any stream capture
// (the look-up is a runtime call that a capture does not allow). The address is cached per
// device index and is not refreshed: do not call this entry point again on a device after
// cudaDeviceReset (or any other teardown of its primary context) in the same process.
//
// All calls share the array and each call overwrites every element it reads before reading it,
// so no zeroing is needed; calls that overlap on the GPU (two streams, two threads, or two
// devices' worth of work enqueued on one device concurrently) race on it.
#include <mutex>

#include "internal.h"

namespace {

// 48 MiB: enough for the H50 workload (T: 3.75e6, b: 1.25e6, d: 2.5e4 doubles).
constexpr long long kStaticScratchDoubles = 48ll * 1024 * 1024 / 8;
__device__ __align__(256) double g_jk_scratch[kStaticScratchDoubles];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// d^P_p = b^P_pp
__global__ void k_static_diag(const double* b, int X, int a, double* d) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)X * a) return;
    long long P = idx / a;
    int p = (int)(idx % a);
    d[idx] = b[P * a * a + (long long)p * a + p];
}

// K_pq = sum_P (b^P_pq)^2
__global__ void k_static_ksum(const double* b, int X, int a, double* K) {
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

// Device address of the scratch array for the current device (looked up once per device).
int static_scratch(double** out) {
    int dev = 0;
    NOF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        nof_set_error("nof_jk_static: device index out of range");
        return NOF_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        double* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void**)&p, g_jk_scratch);
        if (e != cudaSuccess || !p) return nof_cuda_fail(e, "cudaGetSymbolAddress(g_jk_scratch)", __FILE__, __LINE__);
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return NOF_OK;
}

}  // namespace

extern "C" int nof_jk_static(int naux, int nbf, int nact, const double* B, const double* C, double* J,
                             double* K, void* stream) {
    if (naux <= 0 || nbf <= 0 || nact <= 0 || nact > nbf || !B || !C || !J || !K) {
        nof_set_error("nof_jk_static: bad sizes or null pointer");
        return NOF_EINVAL;
    }
    const long long X = naux, n = nbf, a = nact;
    const long long need = X * n * a + X * a * a + X * a;
    if (need > kStaticScratchDoubles) {
        nof_set_error("nof_jk_static: naux*nbf*nact + naux*nact*(nact+1) = " + std::to_string(need) +
                      " doubles exceeds the fixed scratch of " + std::to_string(kStaticScratchDoubles) +
                      " doubles (48 MiB)");
        return NOF_EINVAL;
    }
    // launch-shape limits of the FP64 GEMMs below (64-row tiles of the X n rows of the half
    // transform and one batch entry per aux function of the full transform in grid.y / grid.z),
    // checked before anything is queued so that a refused call leaves no partial work behind
    if (X > 65535 || (X * n + 63) / 64 > 65535) {
        nof_set_error("nof_jk_static: naux = " + std::to_string(X) + " and naux*nbf = " + std::to_string(X * n) +
                      " must stay within 65535 and 65535*64 (grid limits of the transforms)");
        return NOF_EINVAL;
    }
    double* scratch = nullptr;
    NOF_TRY(static_scratch(&scratch));
    double* T = scratch;           // [X][n][a]
    double* b = T + X * n * a;     // [X][a][a]
    double* d = b + X * a * a;     // [X][a]
    cudaStream_t st = (cudaStream_t)stream;
    {   // T[P][mu][p] = sum_nu B[P][mu][nu] C[nu][p]
        Gemm64 g;
        g.M = (int)(X * n); g.N = (int)a; g.K = (int)n;
        g.A = B; g.sAm = n; g.sAk0 = 1;
        g.B = C; g.sBn = 1; g.sBk0 = n;
        g.C = T; g.sCm = a; g.sCn = 1;
        NOF_TRY(gemm64(g, st));
    }
    {   // b[P][q][p] = sum_mu C[mu][q] T[P][mu][p]
        Gemm64 g;
        g.M = (int)a; g.N = (int)a; g.K = (int)n; g.batch = (int)X;
        g.A = C; g.sAm = 1; g.sAk0 = n;
        g.B = T; g.sBn = 1; g.sBk0 = a; g.bB = n * a;
        g.C = b; g.sCm = a; g.sCn = 1; g.bC = a * a;
        NOF_TRY(gemm64(g, st));
    }
    k_static_diag<<<(unsigned)((X * a + 255) / 256), 256, 0, st>>>(b, (int)X, (int)a, d);
    NOF_LAUNCH_CHECK();
    {   // J = d^T d; the free tail of the array holds the split-K partials that gemm64 takes for a
        // small a x a output (summed in a fixed order, so the result does not depend on scheduling)
        Gemm64 g;
        g.M = (int)a; g.N = (int)a; g.K = (int)X;
        g.A = d; g.sAm = 1; g.sAk0 = a;
        g.B = d; g.sBn = 1; g.sBk0 = a;
        g.C = J; g.sCm = a; g.sCn = 1;
        g.work = d + X * a;
        g.work_cap = (size_t)(kStaticScratchDoubles - need);
        NOF_TRY(gemm64(g, st));
    }
    k_static_ksum<<<(unsigned)((a * a + 255) / 256), 256, 0, st>>>(b, (int)X, (int)a, K);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}
