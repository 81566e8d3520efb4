// Exact digit-plane GEMM on the 5th-generation tensor cores (tcgen05 + TMEM + TMA), sm_103a.
//
// Operands are "digit planes": a real matrix X with a power-of-two scale 2^e per row is written
// as X = 2^e sum_{i<4} d_i 256^{-(i+1)} with integer digits |d_0| <= 256, |d_i| <= 128 (i > 0),
// each plane stored as BF16 (integers up to 256 are exact in BF16). For A (M x K) and B (N x K),
//   sum_k A_mk B_nk = 2^{e_m + f_n} 2^{-16} sum_{lvl=0..3} 256^{-lvl} S_lvl,
//   S_lvl = sum_{i+j=lvl} sum_k dA_i[m][k] dB_j[n][k],
// truncated at digit order 3 (10 plane products). Every product is exact and every partial sum
// is an integer below 2^24 as long as one accumulation covers K <= 160, so the FP32 TMEM
// accumulators hold the level sums exactly. The epilogue returns the exact integer
// V = S_0 256^3 + S_1 256^2 + S_2 256 + S_3 (|V| < 2^49), value = 2^{e_m + f_n - 40} V.
//
// Storage ("atom-major"): plane p, K atom t (16 consecutive k), row r, lane j at
// ((p * katoms + t) * rows + r) * 16 + j. A TMA box (16, 128 rows, 2 atoms, 4 planes) lands in
// shared memory as eight 4 KB K-major SWIZZLE_32B atoms, the canonical layout the MMA reads.
//
// Roles (128 threads): warp 0 lane 0 issues TMA, warp 1 lane 0 issues MMAs, all four warps
// drain TMEM (warp w owns lanes 32w..32w+31 = tile rows). Every mbarrier wait is bounded; on
// timeout the kernel sets NOF_DEV_TIMEOUT in the status word, drains what it issued and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "internal.h"
#include "digit_gemm.h"
#include <cuda_bf16.h>
#include <string>

namespace {

constexpr int kBM = 128;
constexpr int kStageAtoms = 2;
constexpr int kStages = 2;
constexpr unsigned long long kTimeoutNs = 4000000000ull;  // 4 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(phase)
        : "memory");
    return ok != 0;
}
// Bounded wait: false (and NOF_DEV_TIMEOUT set) if the phase did not complete in time.
__device__ bool mbar_wait(uint32_t a, uint32_t phase, int* status) {
    unsigned long long t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (mbar_try(a, phase)) return true;
        if ((it & 1023u) == 0u) {
            unsigned long long t = globaltimer();
            if (t0 == 0) t0 = t;
            else if (t - t0 > kTimeoutNs) {
                atomicOr(status, NOF_DEV_TIMEOUT);
                return false;
            }
        }
    }
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
        : "memory");
}
// Shared-memory matrix descriptor: K-major, SWIZZLE_32B atoms of 8 rows x 32 B (SBO = 256 B).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(256 >> 4) << 32;   // stride byte offset between 8-row groups
    d |= (uint64_t)1 << 46;            // descriptor version for tcgen05
    d |= (uint64_t)6 << 61;            // SWIZZLE_32B
    return d;
}
// Instruction descriptor: kind::f16, BF16 x BF16 -> FP32, both K-major, M = 128, N.
__host__ __device__ constexpr uint32_t idesc_bf16(int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// One CTA computes a 128-row x N tile over K atoms [blockIdx.y * katoms, +katoms).
__global__ void __launch_bounds__(128, 2)
k_digit_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
             DigitGemmArgs g) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1 KB alignment for the swizzled atoms
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int N = g.N;
    const uint32_t a_stage_bytes = 4u * kStageAtoms * kBM * 32u;
    const uint32_t b_stage_bytes = 4u * kStageAtoms * (uint32_t)N * 32u;
    unsigned char* sA = smem;
    unsigned char* sB = smem + kStages * a_stage_bytes;
    uint64_t* bars = (uint64_t*)(sB + kStages * b_stage_bytes);  // full[2], empty[2], done
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * kStages + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile_m = blockIdx.x;
    const int katom0 = blockIdx.y * g.katoms;
    const int nk = (g.katoms + kStageAtoms - 1) / kStageAtoms;  // pipeline iterations
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[kStages]),
                   done = smem_u32(&bars[2 * kStages]);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)g.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0 && lane == 0) {
        // TMA producer
        for (int it = 0; it < nk && ok; ++it) {
            int s = it % kStages;
            if (it >= kStages) ok = mbar_wait(empty0 + 8 * s, ((it / kStages) - 1) & 1, g.status);
            if (!ok) break;
            // a TMA box always delivers all kStageAtoms atoms (zero-filled past the tensor end)
            uint32_t bytes = (uint32_t)kStageAtoms * 4u * 32u * (kBM + (uint32_t)N);
            mbar_expect_tx(full0 + 8 * s, bytes);
            int ka = katom0 + it * kStageAtoms;
            tma_load_4d(smem_u32(sA + s * a_stage_bytes), &mapA, 0, tile_m * kBM, ka, 0, full0 + 8 * s);
            tma_load_4d(smem_u32(sB + s * b_stage_bytes), &mapB, 0, 0, ka, 0, full0 + 8 * s);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: level l = i + j accumulates in TMEM columns [l N, (l+1) N)
        const uint32_t idesc = idesc_bf16(N);
        bool started[4] = {false, false, false, false};
        for (int it = 0; it < nk && ok; ++it) {
            int s = it % kStages;
            ok = mbar_wait(full0 + 8 * s, (it / kStages) & 1, g.status);
            if (!ok) break;
            tc_fence_after();
            int atoms = min(kStageAtoms, g.katoms - it * kStageAtoms);
            uint32_t aBase = smem_u32(sA + s * a_stage_bytes), bBase = smem_u32(sB + s * b_stage_bytes);
            for (int t = 0; t < atoms; ++t) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
#pragma unroll
                    for (int j = 0; j < 4 - i; ++j) {
                        int l = i + j;
                        // box layout [plane][atom][rows][16]: plane stride = atoms-in-box * rows * 32 B
                        uint64_t ad = sdesc(aBase + (uint32_t)((i * kStageAtoms + t) * kBM * 32));
                        uint64_t bd = sdesc(bBase + (uint32_t)((j * kStageAtoms + t) * N * 32));
                        mma_bf16(tmem + (uint32_t)(l * N), ad, bd, idesc, started[l] ? 1u : 0u);
                        started[l] = true;
                    }
                }
            }
            mma_commit(empty0 + 8 * s);  // frees the stage once these MMAs retire
        }
        if (ok) mma_commit(done);
    }
    __syncwarp();
    // epilogue: every warp drains its 32 TMEM lanes
    bool ready = mbar_wait(done, 0, g.status);
    tc_fence_after();
    if (ready) {
        const int row = tile_m * kBM + warp * 32 + lane;
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v0[16], v1[16], v2[16], v3[16];
            tmem_ld16(tmem + lane_base + (uint32_t)c0, v0);
            tmem_ld16(tmem + lane_base + (uint32_t)(N + c0), v1);
            tmem_ld16(tmem + lane_base + (uint32_t)(2 * N + c0), v2);
            tmem_ld16(tmem + lane_base + (uint32_t)(3 * N + c0), v3);
            tmem_wait_ld();
            if (row < g.M) {
                long long* orow = g.out + (long long)row * g.ldo;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    int col = c0 + q;
                    if (col >= g.Nvalid) continue;
                    long long V = __float2ll_rn(v0[q]) * 16777216LL + __float2ll_rn(v1[q]) * 65536LL +
                                  __float2ll_rn(v2[q]) * 256LL + __float2ll_rn(v3[q]);
                    if (g.atomic)
                        atomicAdd((unsigned long long*)(orow + col), (unsigned long long)V);
                    else
                        orow[col] = V;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (!ok && threadIdx.x == 0) {
        // a wait gave up: let the copies this CTA issued land before the shared memory goes away
        for (int s = 0; s < kStages; ++s) (void)mbar_wait(full0 + 8 * s, 0, g.status);
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)g.tmem_cols));
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 4-D map over atom-major digit planes: (16 lanes, rows, K atoms, 4 planes), box (16, box_rows,
// stage atoms, 4), SWIZZLE_32B.
int make_map(CUtensorMap* m, const void* base, int rows, int katoms, int box_rows) {
    auto enc = get_encode();
    if (!enc) {
        nof_set_error("cuTensorMapEncodeTiled is unavailable from the driver");
        return NOF_ECUDA;
    }
    cuuint64_t dims[4] = {16, (cuuint64_t)rows, (cuuint64_t)katoms, 4};
    cuuint64_t strides[3] = {32, (cuuint64_t)rows * 32, (cuuint64_t)katoms * rows * 32};
    cuuint32_t box[4] = {16, (cuuint32_t)box_rows, (cuuint32_t)kStageAtoms, 4};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        nof_set_error("cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ")");
        return NOF_ECUDA;
    }
    return NOF_OK;
}

}  // namespace

size_t digit_gemm_smem(int N) {
    return (size_t)kStages * 4 * kStageAtoms * 32 * (kBM + N) + 8 * (2 * kStages + 1) + 16 + 1024;
}

int digit_gemm_plan(DigitGemmPlan* p, const uint16_t* A, int rowsA, const uint16_t* B, int N,
                    int katoms_total, int katoms, int M, int Nvalid, long long* out, long long ldo,
                    bool atomic, int* status) {
    if (N % 16 || N < 16 || N > 128 || katoms < 1 || katoms > 10 || katoms_total % katoms || M <= 0 ||
        Nvalid > N || rowsA < M) {
        nof_set_error("digit_gemm: unsupported shape");
        return NOF_EINVAL;
    }
    NOF_TRY(make_map(&p->ma, A, rowsA, katoms_total, kBM));
    NOF_TRY(make_map(&p->mb, B, N, katoms_total, N));
    DigitGemmArgs& g = p->g;
    g.M = M; g.N = N; g.Nvalid = Nvalid; g.katoms = katoms;
    g.out = out; g.ldo = ldo; g.atomic = atomic ? 1 : 0; g.status = status;
    int cols = 32;
    while (cols < 4 * N) cols *= 2;
    g.tmem_cols = cols;
    p->smem = digit_gemm_smem(N);
    p->grid = dim3((M + kBM - 1) / kBM, katoms_total / katoms);
    static bool attr_done = false;
    if (!attr_done) {
        NOF_CUDA(cudaFuncSetAttribute(k_digit_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)digit_gemm_smem(128)));
        attr_done = true;
    }
    return NOF_OK;
}

int digit_gemm_run(const DigitGemmPlan& p, cudaStream_t st) {
    k_digit_gemm<<<p.grid, 128, p.smem, st>>>(p.ma, p.mb, p.g);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

// A: atom-major planes with rowsA rows (>= M), B: atom-major planes with N rows (padded N),
// both with katoms_total K atoms. K range per CTA: katoms (split-K chunks = katoms_total/katoms).
int digit_gemm(const uint16_t* A, int rowsA, const uint16_t* B, int N, int katoms_total, int katoms,
               int M, int Nvalid, long long* out, long long ldo, bool atomic, int* status,
               cudaStream_t st) {
    DigitGemmPlan p;
    NOF_TRY(digit_gemm_plan(&p, A, rowsA, B, N, katoms_total, katoms, M, Nvalid, out, ldo, atomic, status));
    return digit_gemm_run(p, st);
}

// ---------------------------------------------------------------------------------------
// Self-test: random digit planes, tcgen05 result vs a SIMT integer reference (must be equal).
// ---------------------------------------------------------------------------------------
namespace {

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
    return x;
}
// plane 0 digits in [-256, 256], others in [-128, 128]; rows >= valid_rows are zero
__global__ void k_random_digits(uint16_t* P, int rows, int valid_rows, int katoms, uint32_t seed) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long per_plane = (long long)katoms * rows * 16;
    if (idx >= 4 * per_plane) return;
    int plane = (int)(idx / per_plane);
    long long rem = idx - plane * per_plane;
    int r = (int)((rem / 16) % rows);
    int range = plane == 0 ? 513 : 257;
    int v = (int)(hash32((uint32_t)idx * 2654435761u + seed) % (uint32_t)range) - range / 2;
    if (r >= valid_rows) v = 0;
    __nv_bfloat16 b = __int2bfloat16_rn(v);
    P[idx] = *reinterpret_cast<uint16_t*>(&b);
}
__device__ __forceinline__ int digit_at(const uint16_t* P, int rows, int katoms, int plane, int r, int k) {
    uint16_t u = P[(((long long)plane * katoms + k / 16) * rows + r) * 16 + (k & 15)];
    __nv_bfloat16 b = *reinterpret_cast<__nv_bfloat16*>(&u);
    return (int)__bfloat162float(b);
}
__global__ void k_ref_digit_gemm(const uint16_t* A, int rowsA, const uint16_t* B, int rowsB, int katoms,
                                 int M, int N, long long* out) {
    int m = blockIdx.x * blockDim.x + threadIdx.x, n = blockIdx.y;
    if (m >= M || n >= N) return;
    long long S[4] = {0, 0, 0, 0};
    for (int k = 0; k < katoms * 16; ++k)
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4 - i; ++j)
                S[i + j] += (long long)digit_at(A, rowsA, katoms, i, m, k) * digit_at(B, rowsB, katoms, j, n, k);
    out[(long long)m * N + n] = S[0] * 16777216LL + S[1] * 65536LL + S[2] * 256LL + S[3];
}
__global__ void k_max_absdiff(const long long* a, const long long* b, long long n, unsigned long long* out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    long long d = a[i] - b[i];
    if (d < 0) d = -d;
    atomicMax(out, (unsigned long long)d);
}

}  // namespace

extern "C" int nof_selftest_digit_gemm(int M, int N, int katoms, int splits, unsigned int seed,
                                       long long* max_abs_diff) {
    if (!max_abs_diff || M <= 0 || N <= 0 || N % 16 || katoms <= 0 || splits <= 0 || katoms % splits) {
        nof_set_error("nof_selftest_digit_gemm: bad arguments");
        return NOF_EINVAL;
    }
    int rowsA = (M + 127) / 128 * 128;
    uint16_t *A = nullptr, *B = nullptr;
    long long *C1 = nullptr, *C2 = nullptr;
    unsigned long long* dmax = nullptr;
    int* status = nullptr;
    int r = NOF_OK;
    auto fail = [&](cudaError_t e, const char* w) { r = nof_cuda_fail(e, w, __FILE__, __LINE__); };
    cudaError_t e;
    if ((e = cudaMalloc(&A, 4ull * katoms * rowsA * 16 * 2)) != cudaSuccess) fail(e, "malloc A");
    if (r == NOF_OK && (e = cudaMalloc(&B, 4ull * katoms * N * 16 * 2)) != cudaSuccess) fail(e, "malloc B");
    if (r == NOF_OK && (e = cudaMalloc(&C1, 8ull * M * N)) != cudaSuccess) fail(e, "malloc C1");
    if (r == NOF_OK && (e = cudaMalloc(&C2, 8ull * M * N)) != cudaSuccess) fail(e, "malloc C2");
    if (r == NOF_OK && (e = cudaMalloc(&dmax, 8)) != cudaSuccess) fail(e, "malloc max");
    if (r == NOF_OK && (e = cudaMalloc(&status, 4)) != cudaSuccess) fail(e, "malloc status");
    if (r == NOF_OK) {
        cudaMemset(dmax, 0, 8);
        cudaMemset(status, 0, 4);
        cudaMemset(C1, 0, 8ull * M * N);
        long long na = 4ll * katoms * rowsA * 16, nb = 4ll * katoms * N * 16;
        k_random_digits<<<(unsigned)((na + 255) / 256), 256>>>(A, rowsA, M, katoms, seed);
        k_random_digits<<<(unsigned)((nb + 255) / 256), 256>>>(B, N, N, katoms, seed ^ 0x9e3779b9u);
        r = digit_gemm(A, rowsA, B, N, katoms, katoms / splits, M, N, C1, N, splits > 1, status, 0);
    }
    if (r == NOF_OK) {
        k_ref_digit_gemm<<<dim3((M + 127) / 128, N), 128>>>(A, rowsA, B, N, katoms, M, N, C2);
        k_max_absdiff<<<(unsigned)(((long long)M * N + 255) / 256), 256>>>(C1, C2, (long long)M * N, dmax);
        unsigned long long h = 0;
        int hs = 0;
        if ((e = cudaMemcpy(&h, dmax, 8, cudaMemcpyDeviceToHost)) != cudaSuccess) fail(e, "copy max");
        else if ((e = cudaMemcpy(&hs, status, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) fail(e, "copy status");
        else {
            *max_abs_diff = (long long)h;
            if (hs & NOF_DEV_TIMEOUT) {
                nof_set_error("digit GEMM self-test: a bounded wait timed out");
                r = NOF_ETIMEOUT;
            }
        }
    }
    cudaFree(A); cudaFree(B); cudaFree(C1); cudaFree(C2); cudaFree(dmax); cudaFree(status);
    return r;
}
