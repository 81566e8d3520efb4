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
// Storage: digit_gemm.h's tile-major core-matrix layout, so one pipeline stage (2 K atoms x 4
// planes) of a 128-row tile of A, or of all N rows of B, is one contiguous block that a single
// bulk copy (cp.async.bulk) places in shared memory in the no-swizzle K-major canonical layout
// (core matrices of 8 rows x 16 bytes; 128 bytes between K-adjacent, 256 bytes between
// row-adjacent core matrices).
//
// Every mbarrier wait is bounded; on timeout the kernel sets NOF_DEV_TIMEOUT in the status word,
// lets what it issued land and exits.
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
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(mbar)
        : "memory");
}
// Shared-memory matrix descriptor: K-major, no swizzle; core matrices of 8 rows x 16 bytes,
// 128 bytes between K-adjacent (leading byte offset) and 256 bytes between row-adjacent
// (stride byte offset) core matrices.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;   // leading byte offset: next core matrix along K
    d |= (uint64_t)(256 >> 4) << 32;   // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;            // descriptor version for tcgen05
    return d;                          // swizzle mode 0 (none)
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

// 2^{e} (S0 2^24 + S1 2^16 + S2 2^8 + S3) as a double-float, for level sums S_k that are exact
// integers below 2^24 held in FP32: error-free two-sums, no integer conversions.
__device__ __forceinline__ float2 levels_to_df(float S0, float S1, float S2, float S3, int e) {
    const float a = S0 * 16777216.0f, b = S1 * 65536.0f, c = S2 * 256.0f;
    float h = a + b;
    float bb = h - a;
    float err = (a - (h - bb)) + (b - bb);
    float h2 = h + c;
    bb = h2 - h;
    err += (h - (h2 - bb)) + (c - bb);
    float h3 = h2 + S3;
    bb = h3 - h2;
    err += (h2 - (h3 - bb)) + (S3 - bb);
    const float hi = h3 + err;
    const float lo = err - (hi - h3);
    if (e >= -126 && e <= 127) {
        const float sc = __int_as_float((e + 127) << 23);
        return make_float2(hi * sc, lo * sc);
    }
    return make_float2(ldexpf(hi, e), ldexpf(lo, e));
}

// sum of two double-floats
__device__ __forceinline__ float2 df2_add(float2 a, float2 b) {
    float s = a.x + b.x;
    float bb = s - a.x;
    float e = (a.x - (s - bb)) + (b.x - bb) + a.y + b.y;
    float hi = s + e;
    return make_float2(hi, e - (hi - s));
}

__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

// Persistent, warp-specialised tile loop. Tiles are (128-row block, K chunk) pairs, row block
// fastest. Warp 0 lane 0 streams A and B stages with TMA through a ring of g.stages shared-memory
// slots that carries over from one tile to the next; warp 1 lane 0 issues the 10 digit-product
// MMAs per K atom into one of g.nbuf TMEM accumulator sets (4 levels x N columns each); warps
// 2..5 drain a finished set (lanes 32*(w%4)..+31), hand it back, and write the exact int64 result.
// With two sets the drain of tile i overlaps the MMAs of tile i + 1.
constexpr int kEpiWarps = 8;  // two per TMEM lane group, each owning half of the columns

__global__ void __launch_bounds__(64 + 32 * kEpiWarps, 1)
k_digit_gemm(const uint16_t* __restrict__ A, const uint16_t* __restrict__ B, DigitGemmArgs g) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int N = g.N, S = g.stages, NB = g.nbuf;
    const uint32_t a_stage_bytes = 4u * kStageAtoms * kBM * 32u;
    const uint32_t b_stage_bytes = 4u * kStageAtoms * (uint32_t)N * 32u;
    unsigned char* sA = smem;
    unsigned char* sB = smem + S * a_stage_bytes;
    uint64_t* bars = (uint64_t*)(sB + S * b_stage_bytes);  // full[S] empty[S] tfull[2] tempty[2]
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * S + 4);
    // per epilogue warp: 32 rows x 16 double-floats (+1 pad) to turn row-per-thread results into
    // coalesced row segments
    float2* stage_out = (float2*)(((uintptr_t)(tmem_slot + 4) + 15) & ~(uintptr_t)15);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[S]),
                   tfull0 = smem_u32(&bars[2 * S]), tempty0 = smem_u32(&bars[2 * S + 2]);
    const int ntiles = g.tiles_m * g.kchunks;
    const int nk = (g.katoms + kStageAtoms - 1) / kStageAtoms;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull0 + 8 * b, 1);
            mbar_init(tempty0 + 8 * b, kEpiWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)g.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            int it = 0;
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                const int tm = tile % g.tiles_m, kc = tile / g.tiles_m;
                for (int st = 0; st < nk && ok; ++st, ++it) {
                    const int s = it % S;
                    if (it >= S) ok = mbar_wait(empty0 + 8 * s, ((it / S) - 1) & 1, g.status);
                    if (!ok) break;
                    const int ka = kc * g.katoms + st * kStageAtoms;
                    const int atoms = min(kStageAtoms, g.katoms - st * kStageAtoms);
                    const uint32_t abytes = (uint32_t)atoms * 4u * kBM * 32u;
                    const uint32_t bbytes = (uint32_t)atoms * 4u * (uint32_t)N * 32u;
                    mbar_expect_tx(full0 + 8 * s, abytes + bbytes);
                    bulk_load(smem_u32(sA + s * a_stage_bytes),
                              A + digit_offset(kBM, g.katoms_total, (long long)tm * kBM, (long long)ka * 16, 0),
                              abytes, full0 + 8 * s);
                    bulk_load(smem_u32(sB + s * b_stage_bytes),
                              B + digit_offset(N, g.katoms_total, 0, (long long)ka * 16, 0), bbytes,
                              full0 + 8 * s);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            const uint32_t idesc = idesc_bf16(N);
            int it = 0, local = 0;
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++local) {
                const int b = local % NB, use = local / NB;
                if (use > 0) ok = mbar_wait(tempty0 + 8 * b, (use - 1) & 1, g.status);
                if (!ok) break;
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(b * g.kparts * 4 * N);
                uint32_t started = 0u;  // bit (part * 4 + level): accumulator already initialised
                for (int st = 0; st < nk && ok; ++st, ++it) {
                    const int s = it % S;
                    ok = mbar_wait(full0 + 8 * s, (it / S) & 1, g.status);
                    if (!ok) break;
                    tc_fence_after();
                    const int atoms = min(kStageAtoms, g.katoms - st * kStageAtoms);
                    const uint32_t aBase = smem_u32(sA + s * a_stage_bytes), bBase = smem_u32(sB + s * b_stage_bytes);
                    for (int t = 0; t < atoms; ++t) {
                        const int part = (st * kStageAtoms + t) / g.apart;
                        const uint32_t pacc = acc + (uint32_t)(part * 4 * N);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
#pragma unroll
                            for (int j = 0; j < 4 - i; ++j) {
                                const int l = i + j;
                                const uint32_t bit = 1u << (part * 4 + l);
                                // stage block order [atom][plane][rows x 16]
                                uint64_t ad = sdesc(aBase + (uint32_t)((t * 4 + i) * kBM * 32));
                                uint64_t bd = sdesc(bBase + (uint32_t)((t * 4 + j) * N * 32));
                                mma_bf16(pacc + (uint32_t)(l * N), ad, bd, idesc, (started & bit) ? 1u : 0u);
                                started |= bit;
                            }
                        }
                    }
                    mma_commit(empty0 + 8 * s);
                }
                if (ok) mma_commit(tfull0 + 8 * b);
            }
        }
    } else {  // epilogue warps 2..2+kEpiWarps-1: lane group q, column half h
        const int q = warp & 3;
        const int h = (warp - 2) / 4;
        // column halves for N >= 32 (a chunk may run up to 7 columns past its half, still inside
        // the allocation); for N = 16 the second warp of each lane group has no columns
        const int cbeg = N >= 32 ? h * (N / 2) : 0;
        const int cend = N >= 32 ? cbeg + N / 2 : (h ? 0 : N);
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int local = 0;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++local) {
            const int b = local % NB, use = local / NB;
            ok = mbar_wait(tfull0 + 8 * b, use & 1, g.status);
            if (!ok) break;
            tc_fence_after();
            const int tm = tile % g.tiles_m;
            const int row = tm * kBM + q * 32 + lane;
            long long* orow = g.out + (long long)row * g.ldo;
            const uint32_t acc = tmem + lane_base + (uint32_t)(b * g.kparts * 4 * N);
            float2* st = stage_out + (warp - 2) * 32 * 17;  // this warp's 32 x 16 (+1) staging tile
            long long* stI = reinterpret_cast<long long*>(st);
            for (int c0 = cbeg; c0 < cend; c0 += 16) {
                const int cw = min(16, cend - c0);  // columns of this chunk owned by the warp
                // the K parts are summed in the staging tile: exactly as int64, or as double-floats
                const int er = (g.outf && row < g.M) ? g.erow[row] - 40 : 0;
                for (int part = 0; part < g.kparts; ++part) {
                    float v0[16], v1[16], v2[16], v3[16];
                    const uint32_t pacc = acc + (uint32_t)(part * 4 * N);
                    tmem_ld16(pacc + (uint32_t)c0, v0);
                    tmem_ld16(pacc + (uint32_t)(N + c0), v1);
                    tmem_ld16(pacc + (uint32_t)(2 * N + c0), v2);
                    tmem_ld16(pacc + (uint32_t)(3 * N + c0), v3);
                    tmem_wait_ld();
                    if (!g.outf) {
                        // level sums are exact integers below 2^24: 32-bit conversions and a 64-bit
                        // integer sum (64-bit int <-> float conversions run at the FP64 rate here)
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const long long Vp = ((long long)__float2int_rn(v0[j]) << 24) +
                                                 ((long long)__float2int_rn(v1[j]) << 16) +
                                                 ((long long)__float2int_rn(v2[j]) << 8) + (long long)__float2int_rn(v3[j]);
                            stI[lane * 17 + j] = part ? stI[lane * 17 + j] + Vp : Vp;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const float2 x = levels_to_df(v0[j], v1[j], v2[j], v3[j], er + g.ecol[min(c0 + j, N - 1)]);
                            st[lane * 17 + j] = part ? df2_add(st[lane * 17 + j], x) : x;
                        }
                    }
                }
                if (!g.outf) {
                    if (row < g.M) {
                        const int lim = min(cend, g.Nvalid);  // columns owned by this warp
                        const long long* V = stI + lane * 17;
                        if (g.atomic) {
                            for (int j = 0; j < 16; ++j)
                                if (c0 + j < lim) atomicAdd((unsigned long long*)(orow + c0 + j), (unsigned long long)V[j]);
                        } else {
                            for (int j = 0; j < 16; ++j)
                                if (c0 + j < lim) orow[c0 + j] = V[j];
                        }
                    }
                } else {
                    // write as whole 128-byte row segments (4 lanes per row, 8 rows per pass)
                    __syncwarp();
                    const int rbase = tm * kBM + q * 32;
#pragma unroll
                    for (int it2 = 0; it2 < 4; ++it2) {
                        const int rr = it2 * 8 + (lane >> 2);
                        const int cc = (lane & 3) * 4;
                        const int grow = rbase + rr;
                        if (cc >= cw) continue;
                        if (grow < g.M && c0 + cc + 3 < g.Nvalid && cc + 3 < cw) {
                            float2* dst = g.outf + (long long)grow * g.ldo + c0 + cc;
                            const float2* src = st + rr * 17 + cc;
                            reinterpret_cast<float4*>(dst)[0] = make_float4(src[0].x, src[0].y, src[1].x, src[1].y);
                            reinterpret_cast<float4*>(dst)[1] = make_float4(src[2].x, src[2].y, src[3].x, src[3].y);
                        } else if (grow < g.M) {
                            for (int u = 0; u < 4; ++u)
                                if (c0 + cc + u < g.Nvalid && cc + u < cw)
                                    g.outf[(long long)grow * g.ldo + c0 + cc + u] = st[rr * 17 + cc + u];
                        }
                    }
                }
                __syncwarp();
            }
            // every TMEM read of this set is complete: hand it back to the MMA warp
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty0 + 8 * b);
        }
    }
    __syncwarp();
    if (!ok) {
        // a wait gave up: give the copies and MMAs this CTA issued time to land (bounded) before
        // the shared memory and TMEM go away
        unsigned long long t0 = globaltimer();
        while (globaltimer() - t0 < 200000ull) __nanosleep(1000);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)g.tmem_cols));
    }
}

}  // namespace

static int stages_for(int N) { return N > 64 ? 2 : 3; }

size_t digit_gemm_smem(int N) {
    return (size_t)stages_for(N) * 4 * kStageAtoms * 32 * (kBM + N) + 8 * (2 * stages_for(N) + 4) + 16 + 16 +
           kEpiWarps * 32 * 17 * sizeof(float2) + 1024;
}

int digit_gemm_plan(DigitGemmPlan* p, const uint16_t* A, const uint16_t* B, int N, int katoms_total,
                    int katoms, int M, int Nvalid, long long* out, long long ldo, bool atomic, int* status) {
    const int kparts = (katoms + 9) / 10;
    if (N % 16 || N < 16 || N > 128 || katoms < 1 || katoms_total % katoms || M <= 0 || Nvalid > N ||
        kparts * 4 * N > 512) {
        nof_set_error("digit_gemm: unsupported shape");
        return NOF_EINVAL;
    }
    p->A = A;
    p->B = B;
    DigitGemmArgs& g = p->g;
    g.outf = nullptr;
    g.erow = nullptr;
    g.ecol = nullptr;
    g.M = M; g.N = N; g.Nvalid = Nvalid; g.katoms = katoms; g.katoms_total = katoms_total;
    g.out = out; g.ldo = ldo; g.atomic = atomic ? 1 : 0; g.status = status;
    g.stages = stages_for(N);
    g.kparts = kparts;
    g.apart = (katoms + kparts - 1) / kparts;
    g.nbuf = (2 * kparts * 4 * N <= 512) ? 2 : 1;
    g.tiles_m = (M + kBM - 1) / kBM;
    g.kchunks = katoms_total / katoms;
    int cols = 32;
    while (cols < g.nbuf * kparts * 4 * N) cols *= 2;
    g.tmem_cols = cols;
    p->smem = digit_gemm_smem(N);
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        NOF_CUDA(cudaGetDevice(&dev));
        NOF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        NOF_CUDA(cudaFuncSetAttribute(k_digit_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    }
    if (p->smem > 220 * 1024) {
        nof_set_error("digit_gemm: shared memory plan too large");
        return NOF_EINVAL;
    }
    const int ntiles = g.tiles_m * g.kchunks;
    p->grid = dim3(ntiles < sms ? ntiles : sms, 1);
    return NOF_OK;
}

int digit_gemm_plan_scaled(DigitGemmPlan* p, const uint16_t* A, const uint16_t* B, int N, int katoms, int M,
                           int Nvalid, float2* out, long long ldo, const int* erow, const int* ecol, int* status) {
    if (ldo & 1) {
        nof_set_error("digit_gemm: the scaled output needs an even leading dimension");
        return NOF_EINVAL;
    }
    NOF_TRY(digit_gemm_plan(p, A, B, N, katoms, katoms, M, Nvalid, nullptr, ldo, false, status));
    p->g.outf = out;
    p->g.erow = erow;
    p->g.ecol = ecol;
    return NOF_OK;
}

int digit_gemm_run(const DigitGemmPlan& p, cudaStream_t st) {
    k_digit_gemm<<<p.grid, 64 + 32 * kEpiWarps, p.smem, st>>>(p.A, p.B, p.g);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

// A: digit planes with M rows (tiles of 128), B: digit planes with N rows (one tile), both with
// katoms_total K atoms. Each tile accumulates katoms atoms (split-K chunks = katoms_total/katoms).
int digit_gemm(const uint16_t* A, const uint16_t* B, int N, int katoms_total, int katoms, int M,
               int Nvalid, long long* out, long long ldo, bool atomic, int* status, cudaStream_t st) {
    DigitGemmPlan p;
    NOF_TRY(digit_gemm_plan(&p, A, B, N, katoms_total, katoms, M, Nvalid, out, ldo, atomic, status));
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
// element (row r, k, plane) of a digit tensor: plane 0 digits in [-256, 256], others in
// [-128, 128]; rows >= valid_rows are zero
__global__ void k_random_digits(uint16_t* P, int RT, int rows_pad, int valid_rows, int katoms, uint32_t seed) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long per_plane = (long long)rows_pad * katoms * 16;
    if (idx >= 4 * per_plane) return;
    int plane = (int)(idx / per_plane);
    long long rem = idx - plane * per_plane;
    long long r = rem / (katoms * 16);
    long long k = rem - r * (katoms * 16);
    int range = plane == 0 ? 513 : 257;
    int v = (int)(hash32((uint32_t)idx * 2654435761u + seed) % (uint32_t)range) - range / 2;
    if (r >= valid_rows) v = 0;
    __nv_bfloat16 b = __int2bfloat16_rn(v);
    P[digit_offset(RT, katoms, r, k, plane)] = *reinterpret_cast<uint16_t*>(&b);
}
__device__ __forceinline__ int digit_at(const uint16_t* P, int RT, int katoms, int plane, int r, int k) {
    uint16_t u = P[digit_offset(RT, katoms, r, k, plane)];
    __nv_bfloat16 b = *reinterpret_cast<__nv_bfloat16*>(&u);
    return (int)__bfloat162float(b);
}
__global__ void k_ref_digit_gemm(const uint16_t* A, const uint16_t* B, int NB, int katoms, int M, int N,
                                 long long* out) {
    int m = blockIdx.x * blockDim.x + threadIdx.x, n = blockIdx.y;
    if (m >= M || n >= N) return;
    long long S[4] = {0, 0, 0, 0};
    for (int k = 0; k < katoms * 16; ++k)
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4 - i; ++j)
                S[i + j] += (long long)digit_at(A, 128, katoms, i, m, k) * digit_at(B, NB, katoms, j, n, k);
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
    const long long na = digit_elems(128, M, katoms), nb = digit_elems(N, N, katoms);
    uint16_t *A = nullptr, *B = nullptr;
    long long *C1 = nullptr, *C2 = nullptr;
    unsigned long long* dmax = nullptr;
    int* status = nullptr;
    int r = NOF_OK;
    auto fail = [&](cudaError_t e, const char* w) { r = nof_cuda_fail(e, w, __FILE__, __LINE__); };
    cudaError_t e;
    if ((e = cudaMalloc(&A, 2ull * na)) != cudaSuccess) fail(e, "malloc A");
    if (r == NOF_OK && (e = cudaMalloc(&B, 2ull * nb)) != cudaSuccess) fail(e, "malloc B");
    if (r == NOF_OK && (e = cudaMalloc(&C1, 8ull * M * N)) != cudaSuccess) fail(e, "malloc C1");
    if (r == NOF_OK && (e = cudaMalloc(&C2, 8ull * M * N)) != cudaSuccess) fail(e, "malloc C2");
    if (r == NOF_OK && (e = cudaMalloc(&dmax, 8)) != cudaSuccess) fail(e, "malloc max");
    if (r == NOF_OK && (e = cudaMalloc(&status, 4)) != cudaSuccess) fail(e, "malloc status");
    if (r == NOF_OK) {
        cudaMemset(dmax, 0, 8);
        cudaMemset(status, 0, 4);
        cudaMemset(C1, 0, 8ull * M * N);
        k_random_digits<<<(unsigned)((na + 255) / 256), 256>>>(A, 128, rowsA, M, katoms, seed);
        k_random_digits<<<(unsigned)((nb + 255) / 256), 256>>>(B, N, N, N, katoms, seed ^ 0x9e3779b9u);
        r = digit_gemm(A, B, N, katoms, katoms / splits, M, N, C1, N, splits > 1, status, 0);
    }
    if (r == NOF_OK) {
        k_ref_digit_gemm<<<dim3((M + 127) / 128, N), 128>>>(A, B, N, katoms, M, N, C2);
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
