// Exact digit-plane GEMM on the 5th-generation tensor cores (tcgen05 + TMEM, bulk copies), sm_103a.
//
// Operands are "digit planes": a real matrix X with a power-of-two scale 2^e per row is written
// as X = 2^e sum_{i<nd} d_i 256^{-(i+1)} with integer digits |d_i| <= 128 for i > 0 and
// |d_0| <= digit_top(nd) (128 with nd = 5, where the scale leaves one bit of headroom; 256 with
// nd = 4), nd = 4 or 5, each plane stored as BF16 (integers up to 256 are exact in BF16). For
// A (M x K) and B (N x K),
//   sum_k A_mk B_nk = 2^{e_m + f_n} 2^{-16} sum_{lvl<nd} 256^{-lvl} S_lvl,
//   S_lvl = sum_{i+j=lvl} sum_k dA_i[m][k] dB_j[n][k],
// truncated at digit order nd - 1 (10 plane products for nd = 4, 15 for nd = 5), a truncation of
// relative order 256^{1-nd}. Every product is an exact integer. The FP32 TMEM accumulators hold
// the sums of the leading levels 0 .. nd - 3 exactly: one accumulation ("part") covers at most
// digit_part_atoms_max(nd) K atoms (20 with 5 digits, 16 with 4), over which those levels stay
// integers below 2^24. The last two levels, weighted 256^{2-nd} and 256^{1-nd} relative to level
// 0, may round once a part's sum passes 2^24 (an error near 2^-40 relative with 5 digits and 2^-32
// with 4, the order of the truncation); their sums stay below 2^31. The epilogue returns
// V = sum_l S_l 256^{nd-1-l} (exact in the leading levels), value 2^{e_m + f_n - 8 (nd + 1)} V.
// Output modes: the int64 V (stored, or added atomically for split-K), the scaled value as
// a double-float, or, when each row of A and B carries its own scale on every part of K
// (part_atoms atoms), the sum over parts of 2^{e_m,part + f_n,part - 8 (nd + 1)} V_part as FP64
// (added atomically, or stored per K chunk for a fixed-order reduction).
//
// Storage: digit_gemm.h's tile-major swizzled layout, so one pipeline stage (2 K atoms x 4
// planes) of a 128-row tile of A, or of a BN-row tile of B, is one contiguous block that a single
// bulk copy (cp.async.bulk) places in shared memory in the 32-byte-swizzled K-major canonical
// layout (rows of 32 bytes, 16-byte halves swapped on rows with bit 2 set, 8-row groups 256
// bytes apart).
//
// Every mbarrier wait is bounded; on timeout the kernel sets NOF_DEV_TIMEOUT in the status word,
// lets what it issued land and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>

#include "internal.h"
#include "digit_gemm.h"
#include <cuda_bf16.h>
#include <mutex>
#include <string>
#include <vector>

namespace {

constexpr int kBM = 128;
constexpr int kStageAtoms = 2;
constexpr unsigned long long kTimeoutNs = 4000000000ull;  // default limit of one wait: 4 s

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
__device__ bool mbar_wait(uint32_t a, uint32_t phase, int* status, unsigned long long limit_ns) {
    unsigned long long t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (mbar_try(a, phase)) return true;
        if ((it & 1023u) == 0u) {
            unsigned long long t = globaltimer();
            if (t0 == 0) t0 = t;
            else if (t - t0 > limit_ns) {
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
// Shared-memory matrix descriptor: K-major with 32-byte swizzling (layout type 6); rows of
// 32 bytes (one K atom), 8-row groups 256 bytes apart (stride byte offset); the leading byte
// offset is unused for swizzled K-major operands (1 by convention).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;            // leading byte offset (unused)
    d |= (uint64_t)(256 >> 4) << 32;   // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;            // descriptor version for tcgen05
    d |= (uint64_t)6 << 61;            // swizzle: 32 bytes
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
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// x 2^e for a double-float x, as (x 2^{e1}) 2^{e2} with e1 = floor(e / 2), e2 = e - e1: once e is
// clamped to [-252, 252] both factors are normal powers of two. The intermediate lies between x
// and the result, so every normal result is exact, the same as with ldexpf (only subnormal
// results can round twice); beyond the clamp every nonzero result is 0 or infinite either way.
// No branch and no library call per element.
__device__ __forceinline__ float2 scale_df(float2 x, int e) {
    e = min(max(e, -252), 252);
    const int e1 = e >> 1, e2 = e - e1;
    const float s1 = __int_as_float((e1 + 127) << 23), s2 = __int_as_float((e2 + 127) << 23);
    return make_float2((x.x * s1) * s2, (x.y * s1) * s2);
}

// 2^{e} sum_l S_l 256^{ND-1-l} as a double-float, for level sums S_l that are exact integers
// below 2^24 held in FP32: each scaled level is exact, and error-free two-sums collect the total
// (no integer conversions).
template <int ND>
__device__ __forceinline__ float2 levels_to_df(const float* S, int e) {
    float h = S[0] * (float)(1ull << (8 * (ND - 1)));
    float err = 0.f;
#pragma unroll
    for (int l = 1; l < ND; ++l) {
        const float c = S[l] * (float)(1u << (8 * (ND - 1 - l)));
        const float h2 = h + c;
        const float bb = h2 - h;
        err += (h - (h2 - bb)) + (c - bb);
        h = h2;
    }
    const float hi = h + err;
    return scale_df(make_float2(hi, err - (hi - h)), e);
}

// The int64 V (|V| < 2^63) as a double-float times 2^e: V = a 2^42 + b 2^21 + c with |a| < 2^21
// and 0 <= b, c < 2^21, each exact in FP32 (32-bit conversions; 64-bit ones run at the FP64 rate
// here), collected by error-free two-sums (relative error near 2^-48).
__device__ __forceinline__ float2 int_to_df(long long V, int e) {
    const long long a = V >> 42;
    const long long r = V - (a << 42);
    const float c1 = (float)(int)(r >> 21) * 2097152.0f, c2 = (float)(int)(r & 2097151);
    float h = (float)(int)a * 4398046511104.0f;
    float err = 0.f;
    float h2 = h + c1, bb = h2 - h;
    err += (h - (h2 - bb)) + (c1 - bb);
    h = h2;
    h2 = h + c2;
    bb = h2 - h;
    err += (h - (h2 - bb)) + (c2 - bb);
    h = h2;
    const float hi = h + err;
    return scale_df(make_float2(hi, err - (hi - h)), e);
}

// a double-float in the bits of one 64-bit register (hi in the low word, lo in the high word)
__device__ __forceinline__ long long pack_df(float2 x) {
    return (long long)(((unsigned long long)__float_as_uint(x.y) << 32) | (unsigned long long)__float_as_uint(x.x));
}
__device__ __forceinline__ float2 unpack_df(long long v) {
    const unsigned long long u = (unsigned long long)v;
    return make_float2(__uint_as_float((unsigned)(u & 0xffffffffull)), __uint_as_float((unsigned)(u >> 32)));
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

// Persistent, warp-specialised tile loop. A tile is (N tile, 128-row block, K chunk), N tile
// fastest so that the CTAs working on the N tiles of one row block at the same time share its A
// stages through L2. A chunk is cut into parts of at most g.apart atoms (one exact accumulation
// each). Warp 0 lane 0 streams A and B stages with bulk copies through a ring of g.stages
// shared-memory slots that carries over from one tile to the next; warp 1 lane 0 issues the
// digit-product MMAs (6 per K atom with 4 digits, 9 with 5: pairs of products share one MMA of
// width 2 BN) of a part into one of g.nbuf TMEM accumulator sets (nd levels x BN columns); the
// epilogue warps drain each finished part into running sums held in registers (exact int64 sums,
// or double-float sums of per-part-scaled values: each lane owns one row and up to 48 columns),
// hand the set back, and after the last part of a tile write their rows (the int64 sums of the
// scaled output converted once; single-part tiles of the scaled output through a small staging
// tile, so that consecutive lanes store along a row). With two sets the drain of one part overlaps
// the MMAs of the next; with one (tiles wider than 48 columns with 5 digits) the MMAs wait for it.
// Tiles go to CTAs round-robin, or, with a tile counter, dynamically: after its first tile
// (blockIdx.x) the producer takes each next tile by a fetch-and-add and hands every index to the
// MMA and epilogue warps through a small queue in shared memory. A CTA that starts late (its SM
// still busy with another stream's blocks) then takes fewer tiles instead of holding up the launch.
constexpr int kEpiWarps = 8;  // two per TMEM lane group, each owning half of the columns
// columns of one epilogue warp (BN / 2 for BN >= 32, BN for BN 16), a template parameter MAXC of the
// kernel: 40 for BN <= 80, 48 for BN 96 (whose 48 running sums leave a few registers to spill)
constexpr int kMaxColsOf(int BN) { return BN > 80 ? 48 : 40; }
// the staging tile of one epilogue warp: 32 rows of its columns, an odd pitch in 8-byte words
__host__ __device__ constexpr int stage_pitch(int BN) { return (BN >= 32 ? BN / 2 : 16) + 1; }
constexpr int kTileQ = 4;     // tile-index queue slots (dynamic tiles)


// kPS: per-part scales (the Lagrangian contraction), a separate instantiation so that each output
// mode's epilogue gets the registers to itself
template <int ND, int kMaxCols, bool kPS>
__global__ void __launch_bounds__(64 + 32 * kEpiWarps, 1)
k_digit_gemm(const uint16_t* __restrict__ A, const uint16_t* __restrict__ B, DigitGemmArgs g) {
    // 32-byte swizzling repeats every 256 bytes: every operand block starts on a 256-byte boundary
    extern __shared__ __align__(256) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 255) & ~(uintptr_t)255);
    const int BN = g.BN, S = g.stages, NB = g.nbuf;
    const uint32_t a_stage_bytes = (uint32_t)ND * kStageAtoms * kBM * 32u;
    const uint32_t b_stage_bytes = (uint32_t)ND * kStageAtoms * (uint32_t)BN * 32u;
    unsigned char* sA = smem;
    unsigned char* sB = smem + S * a_stage_bytes;
    // full[S] empty[S] tfull[2] tempty[2] qfull[kTileQ] qempty[kTileQ]
    uint64_t* bars = (uint64_t*)(sB + S * b_stage_bytes);
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * S + 4 + 2 * kTileQ);
    volatile int* tq_id = (volatile int*)(tmem_slot + 4);  // queued tile indices (dynamic tiles)
    // staging tiles of the epilogue warps (g.staged), 16-byte aligned after the queue
    float2* stage_out = (float2*)(((uintptr_t)(tq_id + kTileQ) + 15) & ~(uintptr_t)15);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[S]),
                   tfull0 = smem_u32(&bars[2 * S]), tempty0 = smem_u32(&bars[2 * S + 2]),
                   qfull0 = smem_u32(&bars[2 * S + 4]), qempty0 = smem_u32(&bars[2 * S + 4 + kTileQ]);
    const int ntiles = g.tiles_n * g.tiles_m * g.kchunks;
    const bool dyn = g.tctr != nullptr;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull0 + 8 * b, 1);
            mbar_init(tempty0 + 8 * b, kEpiWarps);
        }
        for (int i = 0; i < kTileQ; ++i) {
            mbar_init(qfull0 + 8 * i, 1);
            mbar_init(qempty0 + 8 * i, 1 + kEpiWarps);  // the MMA warp and every epilogue warp
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
    // the qi-th tile of this CTA for the MMA and epilogue warps: round-robin, or the producer's qi-th
    // queued index, taken by lane 0 (which frees the slot) and passed to the other calling lanes
    // (`lanes`: lane 0 alone for the MMA issuer, the whole warp for an epilogue warp)
    auto consumer_tile = [&](int qi, unsigned lanes) {
        if (!dyn) return (int)blockIdx.x + qi * (int)gridDim.x;
        const int slot = qi % kTileQ;
        int t = ntiles, okl = 1;
        if (lane == 0) {
            okl = mbar_wait(qfull0 + 8 * slot, (qi / kTileQ) & 1, g.status, g.timeout_ns) ? 1 : 0;
            if (okl) {
                t = tq_id[slot];
                mbar_arrive(qempty0 + 8 * slot);
            }
        }
        if (lanes != 1u) {
            t = __shfl_sync(lanes, t, 0);
            okl = __shfl_sync(lanes, okl, 0);
        }
        ok = okl != 0;
        return ok ? t : ntiles;
    };

    if (warp == 0) {
        if (lane == 0) {  // bulk-copy producer
            // dynamic tiles: every CTA starts with tile blockIdx.x (gridDim.x <= ntiles) and takes
            // each further tile as gridDim.x + a fetch-and-add on the launch's counter. Every CTA's
            // run ends with one fetch past the last tile, so a launch makes ntiles fetches; the
            // final one (counter value ntiles - 1) puts the counter back to 0 for the next launch.
            const int last = ntiles + (int)gridDim.x - 1;
            auto fetch = [&]() {
                const int t = (int)gridDim.x + atomicAdd(g.tctr, 1);
                if (t == last) atomicExch(g.tctr, 0);
                return t;
            };
            int it = 0;
            int tile = (int)blockIdx.x;
            for (int qi = 0; ok; ++qi) {
                if (dyn) {  // hand the tile index to the MMA and epilogue warps
                    const int slot = qi % kTileQ;
                    if (qi >= kTileQ) ok = mbar_wait(qempty0 + 8 * slot, ((qi / kTileQ) - 1) & 1, g.status, g.timeout_ns);
                    if (!ok) break;
                    tq_id[slot] = tile;
                    mbar_arrive(qfull0 + 8 * slot);
                }
                if (tile >= ntiles) break;
                const int tn = tile % g.tiles_n, rest = tile / g.tiles_n;
                const int tm = rest % g.tiles_m, kc = rest / g.tiles_m;
                const int k0 = kc * g.katoms, tk = min(g.katoms, g.katoms_total - k0);
                const int nst = (tk + kStageAtoms - 1) / kStageAtoms;
                for (int st = 0; st < nst && ok; ++st, ++it) {
                    const int s = it % S;
                    if (it >= S) ok = mbar_wait(empty0 + 8 * s, ((it / S) - 1) & 1, g.status, g.timeout_ns);
                    if (!ok) break;
                    const int ka = k0 + st * kStageAtoms;
                    const int atoms = min(kStageAtoms, tk - st * kStageAtoms);
                    const uint32_t abytes = (uint32_t)atoms * ND * kBM * 32u;
                    const uint32_t bbytes = (uint32_t)atoms * ND * (uint32_t)BN * 32u;
                    if (g.no_copies) continue;  // failure-detection test: the stage never fills
                    mbar_expect_tx(full0 + 8 * s, abytes + bbytes);
                    // each operand's stage block is one contiguous run of bytes
                    bulk_load(smem_u32(sA + s * a_stage_bytes),
                              A + digit_offset(kBM, g.katoms_total, (long long)tm * kBM, (long long)ka * 16, 0, ND),
                              abytes, full0 + 8 * s);
                    bulk_load(smem_u32(sB + s * b_stage_bytes),
                              B + digit_offset(BN, g.katoms_total, (long long)tn * BN, (long long)ka * 16, 0, ND),
                              bbytes, full0 + 8 * s);
                }
                // the next tile, taken once this one's copies are queued (its latency overlaps
                // the wait for a free ring slot)
                tile = dyn ? fetch() : tile + (int)gridDim.x;
            }
            // a wait gave up: still make this CTA's final fetch, so that the counter returns to 0
            if (dyn && !ok)
                while (tile < ntiles) tile = fetch();
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            // one MMA per digit product pair: A plane i against B planes j and j + 1 at once. The
            // planes of a stage are consecutive BN-row blocks in shared memory and the levels
            // consecutive BN-column blocks in TMEM, so the 2 BN-wide product lands in levels i + j
            // and i + j + 1. An MMA costs the same for every N up to 96 and little more at 128,
            // so pairs halve the MMA count: 6 instead of 10 per K atom with 4 digits, 9 instead
            // of 15 with 5. Each level still receives the same exact integer products.
            const uint32_t idesc = idesc_bf16(BN), idesc2 = idesc_bf16(2 * BN);
            // descriptors of the ring's slot 0; a slot, atom or plane offset is added in 16-byte
            // units straight to the 14-bit address field (shared addresses stay below 2^18)
            const uint64_t adesc0 = sdesc(smem_u32(sA)), bdesc0 = sdesc(smem_u32(sB));
            const uint32_t a_slot16 = a_stage_bytes >> 4, b_slot16 = b_stage_bytes >> 4;
            const uint32_t b_plane16 = (uint32_t)BN * 2u;  // BN rows x 32 bytes
            int it = 0, unit = 0;
            for (int qi = 0; ok; ++qi) {
                const int tile = consumer_tile(qi, 1u);
                if (tile >= ntiles) break;
                const int kc = tile / (g.tiles_n * g.tiles_m);
                const int tk = min(g.katoms, g.katoms_total - kc * g.katoms);
                const int nparts = (tk + g.apart - 1) / g.apart;
                for (int part = 0; part < nparts && ok; ++part, ++unit) {
                    const int b = unit % NB, use = unit / NB;
                    if (use > 0) ok = mbar_wait(tempty0 + 8 * b, (use - 1) & 1, g.status, g.timeout_ns);
                    if (!ok) break;
                    tc_fence_after();
                    uint32_t accl[ND];  // TMEM column of each level of this set
#pragma unroll
                    for (int l = 0; l < ND; ++l) accl[l] = tmem + (uint32_t)((b * ND + l) * BN);
                    const int pa = min(g.apart, tk - part * g.apart);
                    const int nst = (pa + kStageAtoms - 1) / kStageAtoms;
                    for (int st = 0; st < nst && ok; ++st, ++it) {
                        const int s = it % S;
                        ok = mbar_wait(full0 + 8 * s, (it / S) & 1, g.status, g.timeout_ns);
                        if (!ok) break;
                        tc_fence_after();
                        const int atoms = min(kStageAtoms, pa - st * kStageAtoms);
                        const uint64_t ad = adesc0 + (uint64_t)(s * a_slot16);
                        const uint64_t bd = bdesc0 + (uint64_t)(s * b_slot16);
                        // the first product of each level in a part starts its accumulator
                        const uint32_t acc0 = st > 0 ? 1u : 0u;
#pragma unroll
                        for (int t = 0; t < kStageAtoms; ++t) {
                            if (t < atoms) {
                                // stage block order [atom][plane][rows x 16]: plane offsets 256 (A)
                                // and b_plane16 (B) units
                                const uint64_t adt = ad + (uint64_t)(t * ND * 256);
                                const uint64_t bdt = bd + (uint64_t)(t * ND) * b_plane16;
#pragma unroll
                                for (int i = 0; i < ND; ++i) {
#pragma unroll
                                    for (int j = 0; j < ND - i; j += 2) {
                                        const uint32_t accf = (t > 0 || i > 0) ? 1u : acc0;
                                        mma_bf16(accl[i + j], adt + (uint64_t)(i * 256), bdt + (uint64_t)j * b_plane16,
                                                 j + 1 < ND - i ? idesc2 : idesc, accf);
                                    }
                                }
                            }
                        }
                        mma_commit(empty0 + 8 * s);
                    }
                    if (ok) mma_commit(tfull0 + 8 * b);
                }
            }
        }
    } else {  // epilogue warps 2..2+kEpiWarps-1: lane group q, column half h
        const int q = warp & 3;
        const int h = (warp - 2) / 4;
        // column halves for BN >= 32; for BN = 16 the second warp of each lane group has no columns
        const int cbeg = BN >= 32 ? h * (BN / 2) : 0;
        const int cend = BN >= 32 ? cbeg + BN / 2 : (h ? 0 : BN);
        const int cw = cend - cbeg;  // <= kMaxCols
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int unit = 0;
        for (int qi = 0; ok; ++qi) {  // qi: this CTA's tile sequence (q is the lane group)
            const int tile = consumer_tile(qi, 0xffffffffu);
            if (tile >= ntiles) break;
            const int tn = tile % g.tiles_n, rest = tile / g.tiles_n;
            const int tm = rest % g.tiles_m, kc = rest / g.tiles_m;
            const int tk = min(g.katoms, g.katoms_total - kc * g.katoms);
            const int nparts = (tk + g.apart - 1) / g.apart;
            const int rbase = tm * kBM + q * 32;
            const int row = rbase + lane;  // this lane's output row
            const int col0 = tn * BN + cbeg;  // global column of this warp's column 0
            constexpr bool partsc = kPS;
            // exact int64 sums over the parts (the int64 output, and the scaled output when V fits:
            // one conversion to a scaled double-float per tile instead of one per part)
            const bool ints = !partsc && (!g.outf || g.isum);
            constexpr int kOff = 8 * (ND + 1);  // value = 2^{e_row + e_col - 8 (ND + 1)} V
            const int er = (g.outf && row < g.M) ? g.erow[row] - kOff : 0;
            // running sums of this lane's row over the parts, in registers: the int64 V, or the bits
            // of a double-float (hi in the low word, lo in the high word)
            long long acc[kMaxCols];
            for (int part = 0; part < nparts && ok; ++part, ++unit) {
                const int b = unit % NB, use = unit / NB;
                const long long gp = (long long)(kc * g.katoms) / g.apart + part;  // part index along K
                // this part's exponents, loaded before the wait so that their latency overlaps it:
                // the row's, and the columns' (column col0 + lane, and col0 + 32 + lane when the
                // warp has more than 32 columns), handed to the other lanes by shuffles
                const int erp = (partsc && row < g.M) ? g.epA[gp * g.M + row] - kOff : er;
                const int* ec = partsc ? g.epB + gp * g.Nvalid : g.ecol;
                const int ecl = ints ? 0 : ec[min(col0 + lane, g.Nvalid - 1)];
                const int ech = (ints || cw <= 32) ? 0 : ec[min(col0 + 32 + lane, g.Nvalid - 1)];
                ok = mbar_wait(tfull0 + 8 * b, use & 1, g.status, g.timeout_ns);
                if (!ok) break;
                tc_fence_after();
                const uint32_t acct = tmem + lane_base + (uint32_t)(b * ND * BN);
#pragma unroll
                for (int c0 = 0; c0 < kMaxCols; c0 += 8) {  // constant indices keep acc in registers
                    if (c0 >= cw) break;  // cw is a multiple of 8
                    // 8 columns of every level at a time: the register budget of a 10-warp CTA (about
                    // 170 per thread: three warps share a sub-partition's 16K registers) holds up to
                    // 40 running sums and ND x 8 loaded values without spilling (with 48 sums, for
                    // BN 96, ptxas spills 8 to 20 bytes per thread)
                    float v[ND][8];
                    const uint32_t col = (uint32_t)(cbeg + c0);
#pragma unroll
                    for (int l = 0; l < ND; ++l) tmem_ld8(acct + (uint32_t)(l * BN) + col, v[l]);
                    tmem_wait_ld();
                    if (ints) {
                        // the leading level sums are exact integers below 2^24 and the last two stay
                        // below 2^31: 32-bit conversions and a 64-bit integer sum (64-bit int <-> float
                        // conversions run at the FP64 rate here)
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            long long Vp = 0;
#pragma unroll
                            for (int l = 0; l < ND; ++l) Vp += (long long)__float2int_rn(v[l][j]) << (8 * (ND - 1 - l));
                            acc[c0 + j] = part ? acc[c0 + j] + Vp : Vp;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int e =
                                erp + __shfl_sync(0xffffffffu, c0 + j < 32 ? ecl : ech, (c0 + j) & 31);
                            float S[ND];
#pragma unroll
                            for (int l = 0; l < ND; ++l) S[l] = v[l][j];
                            float2 x = levels_to_df<ND>(S, e);
                            if (part) x = df2_add(unpack_df(acc[c0 + j]), x);
                            acc[c0 + j] = pack_df(x);
                        }
                    }
                }
                // every TMEM read of this set is complete: hand it back to the MMA warp
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty0 + 8 * b);
            }
            if (!ok) break;
            const int ncol = min(cw, g.Nvalid - col0);  // valid columns of this warp (warp-uniform)
            if (ints && g.outf) {  // the int64 sums as scaled double-floats, in place
#pragma unroll
                for (int c = 0; c < kMaxCols; ++c) {
                    if (c >= ncol) break;
                    acc[c] = pack_df(int_to_df(acc[c], er + g.ecol[col0 + c]));
                }
            }
            if (!partsc && g.staged && ncol > 0) {
                // single-part tiles: the warp's rows go through its staging tile, and consecutive
                // lanes store along a row (cw / 2 lanes of 16-byte column pairs per row, 32 / that
                // many rows per pass)
                const int SP = stage_pitch(BN);
                float2* st = stage_out + (warp - 2) * 32 * SP;
#pragma unroll
                for (int c = 0; c < kMaxCols; ++c) {
                    if (c >= ncol) break;
                    st[lane * SP + c] = unpack_df(acc[c]);
                }
                __syncwarp();
                const int hp = (cw + 1) / 2;
                const int rpp = 32 / hp, lr = lane / hp, cc = 2 * (lane - lr * hp);
                for (int rr = lr; lr < rpp && rr < 32; rr += rpp) {
                    const int grow = rbase + rr;
                    if (grow >= g.M || cc >= ncol) continue;
                    float2* dst = g.outf + (long long)grow * g.ldo + col0 + cc;  // ldo, col0, cc even
                    const float2 x0 = st[rr * SP + cc];
                    if (cc + 1 < ncol) {
                        const float2 x1 = st[rr * SP + cc + 1];
                        *reinterpret_cast<float4*>(dst) = make_float4(x0.x, x0.y, x1.x, x1.y);
                    } else {
                        *dst = x0;
                    }
                }
                __syncwarp();
            }
            // otherwise each lane writes its own row: 16-byte stores of column pairs (double-floats)
            // or one element at a time (int64, FP64 partials, atomics)
            if (ncol > 0 && row < g.M && (partsc || !g.staged)) {
                if (g.out) {
                    long long* dst = g.out + (long long)row * g.ldo + col0;
#pragma unroll
                    for (int c = 0; c < kMaxCols; ++c) {
                        if (c >= ncol) break;
                        if (g.atomic) atomicAdd((unsigned long long*)(dst + c), (unsigned long long)acc[c]);
                        else dst[c] = acc[c];
                    }
                } else if (g.outd) {
                    double* dst = g.outd + (long long)kc * g.chunk_stride + (long long)row * g.ldo + col0;
#pragma unroll
                    for (int c = 0; c < kMaxCols; ++c) {
                        if (c >= ncol) break;
                        const float2 x = unpack_df(acc[c]);
                        const double v = (double)x.x + (double)x.y;
                        if (g.atomic) atomicAdd(dst + c, v);
                        else dst[c] = v;
                    }
                } else {
                    float2* dst = g.outf + (long long)row * g.ldo + col0;  // ldo and col0 even: 16-byte aligned
#pragma unroll
                    for (int c = 0; c < kMaxCols; c += 2) {
                        if (c >= ncol) break;
                        const float2 x0 = unpack_df(acc[c]);
                        if (c + 1 < ncol) {
                            const float2 x1 = unpack_df(acc[c + 1]);
                            *reinterpret_cast<float4*>(dst + c) = make_float4(x0.x, x0.y, x1.x, x1.y);
                        } else {
                            dst[c] = x0;
                        }
                    }
                }
            }
            // column maxima of |value| per group of rows (GEMM1: per aux function; atomics without a
            // return value: nothing waits). When the warp's valid rows lie in at most four groups,
            // then for each group a transposing butterfly over 32 columns at a time (steps 16, 8,
            // 4, 2, 1: each lane keeps half of its columns and takes the partner's maxima of them;
            // rows of the other group count as 0) leaves lane c with column c's maximum, and one
            // atomic per lane follows: 31 shuffles and one atomic instruction per 32 columns.
            const int g_first = rbase / g.group_rows, g_last = min(rbase + 31, g.M - 1) / g.group_rows;
            const bool few_groups = g_last - g_first <= 3;
            for (int grp = g_first; !partsc && g.outf && g.colmax && ncol > 0 && rbase < g.M && few_groups &&
                                    grp <= g_last;
                 ++grp) {
                const bool mine = row < g.M && row / g.group_rows == grp;
#pragma unroll
                for (int cb = 0; cb < kMaxCols; cb += 32) {
                    if (cb >= ncol) break;
                    float v[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        v[i] = (cb + i < kMaxCols && cb + i < ncol && mine) ? fabsf(unpack_df(acc[cb + i < kMaxCols ? cb + i : 0]).x)
                                                                             : 0.f;
#pragma unroll
                    for (int sft = 16; sft >= 1; sft >>= 1) {
                        const bool up = (lane & sft) != 0;
#pragma unroll
                        for (int i = 0; i < sft; ++i) {
                            const float send = up ? v[i] : v[i + sft];
                            const float keep = up ? v[i + sft] : v[i];
                            v[i] = fmaxf(keep, __shfl_xor_sync(0xffffffffu, send, sft));
                        }
                    }
                    if (cb + lane < ncol)
                        atomicMax(g.colmax + (long long)grp * g.Nvalid + col0 + cb + lane, __float_as_uint(v[0]));
                }
            }
            // otherwise (groups of fewer than 11 rows) a segmented reduction over the lanes: groups are
            // runs of consecutive rows, so after steps 1, 2, 4, 8, 16 that only take a lane's value
            // from a lane of the same group, the first lane of each run holds the run's maximum
            if (!partsc && g.outf && g.colmax && ncol > 0 && rbase < g.M && !few_groups) {
                const int grp = row / g.group_rows;
                unsigned same = 0;
#pragma unroll
                for (int i2 = 0; i2 < 5; ++i2) {
                    const int og = __shfl_down_sync(0xffffffffu, grp, 1 << i2);
                    if (lane + (1 << i2) < 32 && og == grp) same |= 1u << i2;
                }
                const int gprev = __shfl_up_sync(0xffffffffu, grp, 1);
                const bool leader = (lane == 0 || gprev != grp) && row < g.M;
#pragma unroll
                for (int c = 0; c < kMaxCols; ++c) {
                    if (c >= ncol) break;
                    float m = row < g.M ? fabsf(unpack_df(acc[c]).x) : 0.f;
#pragma unroll
                    for (int i2 = 0; i2 < 5; ++i2) {
                        const float o = __shfl_down_sync(0xffffffffu, m, 1 << i2);
                        if (same & (1u << i2)) m = fmaxf(m, o);
                    }
                    if (leader) atomicMax(g.colmax + (long long)grp * g.Nvalid + col0 + c, __float_as_uint(m));
                }
            }
            __syncwarp();
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

constexpr size_t kSmemLimit = 227 * 1024;

// the ring of stages, the barriers, the TMEM address slot, the tile queue and, for staged stores,
// the epilogue warps' staging tiles
size_t smem_bytes(int BN, int stages, int nd, bool staged = false) {
    return (size_t)stages * nd * kStageAtoms * 32 * (kBM + BN) + 8 * (2 * stages + 4 + 2 * kTileQ) + 16 +
           4 * kTileQ + 16 + 256 + (staged ? (size_t)kEpiWarps * 32 * stage_pitch(BN) * sizeof(float2) + 16 : 0);
}

}  // namespace

namespace {
template <bool PS>
int set_smem_limits() {
    NOF_CUDA(cudaFuncSetAttribute(k_digit_gemm<4, 40, PS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
    NOF_CUDA(cudaFuncSetAttribute(k_digit_gemm<5, 40, PS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
    NOF_CUDA(cudaFuncSetAttribute(k_digit_gemm<4, 48, PS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
    NOF_CUDA(cudaFuncSetAttribute(k_digit_gemm<5, 48, PS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
    return NOF_OK;
}
template <bool PS>
void launch_digit_gemm(const DigitGemmPlan& p, cudaStream_t st) {
    const dim3 blk(64 + 32 * kEpiWarps);
    const bool wide = kMaxColsOf(p.g.BN) == 48;
    if (p.g.nd == 5) {
        if (wide) k_digit_gemm<5, 48, PS><<<p.grid, blk, p.smem, st>>>(p.A, p.B, p.g);
        else k_digit_gemm<5, 40, PS><<<p.grid, blk, p.smem, st>>>(p.A, p.B, p.g);
    } else {
        if (wide) k_digit_gemm<4, 48, PS><<<p.grid, blk, p.smem, st>>>(p.A, p.B, p.g);
        else k_digit_gemm<4, 40, PS><<<p.grid, blk, p.smem, st>>>(p.A, p.B, p.g);
    }
}
}  // namespace

int digit_gemm_max_stages(int BN, int nd, bool staged) {
    int s = 2;
    while (s < 8 && smem_bytes(BN, s + 1, nd, staged) <= kSmemLimit) ++s;
    return s;
}

int digit_gemm_plan(DigitGemmPlan* p, const uint16_t* A, const uint16_t* B, int M, int Nvalid, int BN, int nd,
                    int katoms_total, int chunk_atoms, int stages, const DigitGemmOut& o, int* status) {
    const int nout = (o.out != nullptr) + (o.outf != nullptr) + (o.outd != nullptr);
    const bool partsc = o.epA != nullptr;
    if ((nd != 4 && nd != 5) || !digit_bn_ok(BN, nd) || M <= 0 || Nvalid <= 0 || katoms_total < 1 ||
        chunk_atoms < 1 || nout != 1 || (o.outf && ((o.ldo & 1) || !o.erow || !o.ecol || o.atomic)) ||
        o.ldo < Nvalid || (o.colmax && (o.group_rows < 1 || !o.outf)) || (partsc != (o.epB != nullptr)) ||
        (partsc && (!o.outd || o.part_atoms < 2 || (o.part_atoms & 1) || o.part_atoms > digit_part_atoms_max(nd) ||
                    chunk_atoms % o.part_atoms)) ||
        (o.outd && !partsc) ||
        (o.chunk_stride && (!o.outd || o.atomic || o.chunk_stride < (long long)M * o.ldo))) {
        nof_set_error("digit_gemm: unsupported shape or output mode");
        return NOF_EINVAL;
    }
    // the exact int64 result of one output element: per K element |V| <= 65536 256^{nd-1} (1 +
    // 2^-8 + 1.25 2^-16 + ...) < 1.004 * 2^16 * 256^{nd-1}; keep the K sum below 2^63
    const bool v_fits = (double)katoms_total * 16.0 * 1.004 * 65536.0 * std::pow(256.0, nd - 1) <= 9.0e18;
    if (o.out && !v_fits) {
        nof_set_error("digit_gemm: K too long for an exact int64 sum");
        return NOF_EINVAL;
    }
    // single-part tiles of the scaled output write through a staging tile when it leaves a ring of
    // at least 3 stages: their stores, not their one drain, dominate the epilogue
    const int katoms_chunk = chunk_atoms < katoms_total ? chunk_atoms : katoms_total;
    const bool staged = o.outf && katoms_chunk <= digit_part_atoms_max(nd) &&
                        smem_bytes(BN, 3, nd, true) <= kSmemLimit && (stages == 0 || smem_bytes(BN, stages, nd, true) <= kSmemLimit);
    if (stages == 0) stages = digit_gemm_max_stages(BN, nd, staged);
    if (stages < 2 || smem_bytes(BN, stages, nd, staged) > kSmemLimit) {
        nof_set_error("digit_gemm: shared memory plan too large");
        return NOF_EINVAL;
    }
    p->A = A;
    p->B = B;
    DigitGemmArgs& g = p->g;
    g.nd = nd;
    g.M = M;
    g.BN = BN;
    g.tiles_n = (Nvalid + BN - 1) / BN;
    g.Nvalid = Nvalid;
    g.katoms = chunk_atoms < katoms_total ? chunk_atoms : katoms_total;
    g.katoms_total = katoms_total;
    // atoms per part: the per-part scales' length, or as few balanced parts as the exactness of
    // the leading levels allows (an even count: a pipeline stage holds two atoms)
    if (partsc) {
        g.apart = o.part_atoms;
    } else {
        const int amax = digit_part_atoms_max(nd);
        const int nparts = (g.katoms + amax - 1) / amax;
        const int per = (g.katoms + nparts - 1) / nparts;
        g.apart = (per + 1) / 2 * 2;
    }
    g.nbuf = digit_nbuf(BN, nd);
    int cols = 32;
    while (cols < g.nbuf * nd * BN) cols *= 2;
    g.tmem_cols = cols;
    g.out = o.out;
    g.outf = o.outf;
    // (with one part per tile a double-float sum is cheaper than a conversion at the end)
    g.isum = (o.outf && v_fits && g.katoms > g.apart) ? 1 : 0;
    g.outd = o.outd;
    g.chunk_stride = o.chunk_stride;
    g.ldo = o.ldo;
    g.atomic = o.atomic ? 1 : 0;
    g.erow = o.erow;
    g.ecol = o.ecol;
    g.epA = o.epA;
    g.epB = o.epB;
    g.colmax = o.colmax;
    g.group_rows = o.group_rows;
    g.status = status;
    g.timeout_ns = kTimeoutNs;
    g.no_copies = 0;
    g.stages = stages;
    g.tiles_m = (M + kBM - 1) / kBM;
    g.kchunks = (katoms_total + g.katoms - 1) / g.katoms;
    g.tctr = o.tile_counter;
    if (g.kchunks > 1 && !o.atomic && !o.chunk_stride) {
        nof_set_error("digit_gemm: split-K needs an atomic or per-chunk output");
        return NOF_EINVAL;
    }
    p->smem = smem_bytes(BN, stages, nd, staged);
    g.staged = staged ? 1 : 0;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        NOF_CUDA(cudaGetDevice(&dev));
        NOF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        NOF_TRY(set_smem_limits<false>());
        NOF_TRY(set_smem_limits<true>());
    }
    const long long ntiles = (long long)g.tiles_n * g.tiles_m * g.kchunks;
    if (ntiles > 0x7fffffffLL) {
        nof_set_error("digit_gemm: too many tiles");
        return NOF_EINVAL;
    }
    p->grid = dim3((unsigned)(ntiles < sms ? ntiles : sms), 1);
    return NOF_OK;
}

int digit_gemm_run(const DigitGemmPlan& p, cudaStream_t st) {
    if (p.g.epA) launch_digit_gemm<true>(p, st);
    else launch_digit_gemm<false>(p, st);
    NOF_LAUNCH_CHECK();
    return NOF_OK;
}

// ---------------------------------------------------------------------------------------
// Autotuner
// ---------------------------------------------------------------------------------------
namespace {
struct TuneEntry {
    DigitTuneKey key;
    int best;
};
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;
bool same_key(const DigitTuneKey& a, const DigitTuneKey& b) {
    return a.kind == b.kind && a.M == b.M && a.Nvalid == b.Nvalid && a.katoms_total == b.katoms_total &&
           a.extra == b.extra;
}
}  // namespace

// Writes 256 MiB (twice the L2) on `st`, so that the next launch reads its operands from HBM. The
// buffer is allocated once per device and kept for the life of the process.
int l2_flush(cudaStream_t st) {
    static std::mutex mu;
    static std::vector<std::pair<int, void*>> bufs;
    constexpr size_t kFlushBytes = 256ull << 20;
    int dev = 0;
    NOF_CUDA(cudaGetDevice(&dev));
    void* buf = nullptr;
    {
        std::lock_guard<std::mutex> lk(mu);
        for (auto& b : bufs)
            if (b.first == dev) buf = b.second;
        if (!buf) {
            NOF_CUDA(cudaMalloc(&buf, kFlushBytes));
            bufs.push_back({dev, buf});
        }
    }
    NOF_CUDA(cudaMemsetAsync(buf, 0, kFlushBytes, st));
    return NOF_OK;
}

int digit_gemm_pick(const DigitTuneKey& key, const DigitGemmPlan* cands, int ncand, cudaStream_t st, int* best,
                    bool cold) {
    if (ncand < 1) {
        nof_set_error("digit_gemm_pick: no candidates");
        return NOF_EINVAL;
    }
    *best = 0;
    if (ncand == 1) return NOF_OK;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (const TuneEntry& e : g_tune)
            if (same_key(e.key, key) && e.best < ncand) {
                *best = e.best;
                return NOF_OK;
            }
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    NOF_CUDA(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone) return NOF_OK;  // no timing inside a capture
    cudaEvent_t e0, e1;
    NOF_CUDA(cudaEventCreate(&e0));
    NOF_CUDA(cudaEventCreate(&e1));
    float best_ms = 3.0e38f;
    int r = NOF_OK;
    for (int i = 0; i < ncand && r == NOF_OK; ++i) {
        r = digit_gemm_run(cands[i], st);  // warm-up
        float ms = 3.0e38f;
        for (int rep = 0; rep < 3 && r == NOF_OK; ++rep) {
            if (cold) r = l2_flush(st);
            if (r != NOF_OK) break;
            cudaEventRecord(e0, st);
            r = digit_gemm_run(cands[i], st);
            cudaEventRecord(e1, st);
            cudaError_t ce = cudaEventSynchronize(e1);
            if (ce != cudaSuccess) {
                r = nof_cuda_fail(ce, "autotune timing", __FILE__, __LINE__);
                break;
            }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            ms = t < ms ? t : ms;
        }
        if (ms < best_ms) {
            best_ms = ms;
            *best = i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != NOF_OK) return r;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.push_back({key, *best});
    return NOF_OK;
}

// ---------------------------------------------------------------------------------------
// Self-test: random digit planes, tcgen05 result vs a SIMT integer reference (must be equal).
// ---------------------------------------------------------------------------------------
namespace {

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
    return x;
}
// element (row r, k, plane) of a digit tensor with nd planes: leading digits in
// [-digit_top(nd), digit_top(nd)], the others in [-128, 128] (the range the digitisers produce);
// rows >= valid_rows are zero
__global__ void k_random_digits(uint16_t* P, int RT, int rows_pad, int valid_rows, int katoms, int nd,
                                uint32_t seed) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long per_plane = (long long)rows_pad * katoms * 16;
    if (idx >= nd * per_plane) return;
    int plane = (int)(idx / per_plane);
    long long rem = idx - plane * per_plane;
    long long r = rem / (katoms * 16);
    long long k = rem - r * (katoms * 16);
    const int range = plane == 0 ? 2 * digit_top(nd) + 1 : 257;
    int v = (int)(hash32((uint32_t)idx * 2654435761u + seed) % (uint32_t)range) - range / 2;
    if (r >= valid_rows) v = 0;
    __nv_bfloat16 b = __int2bfloat16_rn(v);
    P[digit_offset(RT, katoms, r, k, plane, nd)] = *reinterpret_cast<uint16_t*>(&b);
}
__device__ __forceinline__ int digit_at(const uint16_t* P, int RT, int katoms, int nd, int plane, int r, int k) {
    uint16_t u = P[digit_offset(RT, katoms, r, k, plane, nd)];
    __nv_bfloat16 b = *reinterpret_cast<__nv_bfloat16*>(&u);
    return (int)__bfloat162float(b);
}
// V = sum_{i + j < nd} 256^{nd-1-(i+j)} sum_k dA_i dB_j in int64 (plain loops)
__global__ void k_ref_digit_gemm(const uint16_t* A, const uint16_t* B, int NB, int katoms, int nd, int M, int N,
                                 long long* out) {
    int m = blockIdx.x * blockDim.x + threadIdx.x, n = blockIdx.y;
    if (m >= M || n >= N) return;
    long long S[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < katoms * 16; ++k)
        for (int i = 0; i < nd; ++i)
            for (int j = 0; j < nd - i; ++j)
                S[i + j] += (long long)digit_at(A, 128, katoms, nd, i, m, k) * digit_at(B, NB, katoms, nd, j, n, k);
    long long V = 0;
    for (int l = 0; l < nd; ++l) V = V * 256 + S[l];
    out[(long long)m * N + n] = V;
}
// small random exponents in [-6, 6] (row or column scales of the scaled output modes)
__global__ void k_random_exps(int* e, int n, uint32_t seed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) e[i] = (int)(hash32((uint32_t)i * 2246822519u + seed) % 13u) - 6;
}
// The scaled outputs against the exact V: |value 2^-e - V| must stay below tolV (value = hi + lo of a
// double-float, or an FP64 sum over parts whose scales are all erow[m] + ecol[n]); a larger
// deviation marks the comparison failed by raising the running maximum to 2^62.
__global__ void k_check_scaled(const long long* V, const float2* outf, const double* outd, const int* erow,
                               const int* ecol, int M, int N, int nd, double tolV, unsigned long long* out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)M * N) return;
    const int m = (int)(i / N), n = (int)(i - (long long)m * N);
    const double got = outf ? (double)outf[i].x + (double)outf[i].y : outd[i];
    const double back = ldexp(got, -(erow[m] + ecol[n] - 8 * (nd + 1)));
    if (!(fabs(back - (double)V[i]) <= tolV)) atomicMax(out, 1ull << 62);
}
__global__ void k_max_absdiff(const long long* a, const long long* b, long long n, unsigned long long* out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    long long d = a[i] - b[i];
    if (d < 0) d = -d;
    atomicMax(out, (unsigned long long)d);
}

}  // namespace

extern "C" int nof_selftest_digit_gemm(int M, int N, int bn, int nd, int katoms, int chunk_atoms,
                                       unsigned int seed, long long* max_abs_diff) {
    if (!max_abs_diff || M <= 0 || N <= 0 || (nd != 4 && nd != 5) || !digit_bn_ok(bn, nd) || katoms <= 0 ||
        chunk_atoms <= 0) {
        nof_set_error("nof_selftest_digit_gemm: bad arguments");
        return NOF_EINVAL;
    }
    const int rowsA = (M + 127) / 128 * 128, rowsB = (N + bn - 1) / bn * bn;
    const long long na = digit_elems(128, M, katoms, nd), nb = digit_elems(bn, N, katoms, nd);
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
        k_random_digits<<<(unsigned)((na + 255) / 256), 256>>>(A, 128, rowsA, M, katoms, nd, seed);
        k_random_digits<<<(unsigned)((nb + 255) / 256), 256>>>(B, bn, rowsB, N, katoms, nd, seed ^ 0x9e3779b9u);
        DigitGemmOut o;
        o.out = C1;
        o.ldo = N;
        o.atomic = chunk_atoms < katoms;
        DigitGemmPlan p;
        r = digit_gemm_plan(&p, A, B, M, N, bn, nd, katoms, chunk_atoms, 0, o, status);
        if (r == NOF_OK) r = digit_gemm_run(p, 0);
    }
    const unsigned nblkMN = (unsigned)(((long long)M * N + 255) / 256);
    if (r == NOF_OK) {
        k_ref_digit_gemm<<<dim3((M + 127) / 128, N), 128>>>(A, B, bn, katoms, nd, M, N, C2);
        k_max_absdiff<<<nblkMN, 256>>>(C1, C2, (long long)M * N, dmax);
    }
    // dynamic tiles, twice in a row: the second launch checks that the first left its counter at 0
    int* ctr = nullptr;
    if (r == NOF_OK && (e = cudaMalloc(&ctr, sizeof(int))) != cudaSuccess) fail(e, "malloc counter");
    if (r == NOF_OK) {
        cudaMemset(ctr, 0, sizeof(int));
        DigitGemmOut o;
        o.out = C1;
        o.ldo = N;
        o.atomic = chunk_atoms < katoms;
        o.tile_counter = ctr;
        DigitGemmPlan p;
        r = digit_gemm_plan(&p, A, B, M, N, bn, nd, katoms, chunk_atoms, 0, o, status);
        for (int rep = 0; rep < 2 && r == NOF_OK; ++rep) {
            cudaMemset(C1, 0, 8ull * M * N);
            r = digit_gemm_run(p, 0);
            if (r == NOF_OK) k_max_absdiff<<<nblkMN, 256>>>(C1, C2, (long long)M * N, dmax);
        }
    }
    cudaFree(ctr);
    // the scaled double-float output (row and column exponents), and, when K is whole parts of
    // the per-part scales, the FP64 per-part output with every part's scales equal to the row's
    // and column's: both against the exact V within 2^-38 of the largest |V| the shape allows
    // (far below any wrong exponent or column, far above the double-float rounding)
    if (r == NOF_OK && chunk_atoms >= katoms) {
        int *er = nullptr, *ecl = nullptr, *epA = nullptr, *epB = nullptr;
        float2* outf = nullptr;
        double* outd = nullptr;
        const int patoms = digit_scale_part_atoms(nd);
        const bool parts = katoms % patoms == 0;
        const int nparts = parts ? katoms / patoms : 0;
        if ((e = cudaMalloc(&er, 4ull * M)) != cudaSuccess) fail(e, "malloc erow");
        if (r == NOF_OK && (e = cudaMalloc(&ecl, 4ull * N)) != cudaSuccess) fail(e, "malloc ecol");
        if (r == NOF_OK && (e = cudaMalloc(&outf, 8ull * M * N)) != cudaSuccess) fail(e, "malloc outf");
        if (r == NOF_OK && parts && (e = cudaMalloc(&outd, 8ull * M * N)) != cudaSuccess) fail(e, "malloc outd");
        if (r == NOF_OK && parts && (e = cudaMalloc(&epA, 4ull * M * nparts)) != cudaSuccess) fail(e, "malloc epA");
        if (r == NOF_OK && parts && (e = cudaMalloc(&epB, 4ull * N * nparts)) != cudaSuccess) fail(e, "malloc epB");
        const double tolV = std::ldexp(16.0 * katoms * 1.004 * 65536.0 * std::pow(256.0, nd - 1), -38);
        if (r == NOF_OK) {
            k_random_exps<<<(M + 255) / 256, 256>>>(er, M, seed * 3u + 1u);
            k_random_exps<<<(N + 255) / 256, 256>>>(ecl, N, seed * 5u + 2u);
            for (int q = 0; q < nparts; ++q) {  // every part carries the row's and column's scale
                cudaMemcpy(epA + (size_t)q * M, er, 4ull * M, cudaMemcpyDeviceToDevice);
                cudaMemcpy(epB + (size_t)q * N, ecl, 4ull * N, cudaMemcpyDeviceToDevice);
            }
            DigitGemmOut o;
            o.outf = outf;
            o.ldo = N + (N & 1);  // even leading dimension (16-byte pairs)
            o.erow = er;
            o.ecol = ecl;
            DigitGemmPlan p;
            if (o.ldo == N) {
                r = digit_gemm_plan(&p, A, B, M, N, bn, nd, katoms, katoms, 0, o, status);
                if (r == NOF_OK) r = digit_gemm_run(p, 0);
                if (r == NOF_OK)
                    k_check_scaled<<<nblkMN, 256>>>(C2, outf, nullptr, er, ecl, M, N, nd, tolV, dmax);
            }
            if (r == NOF_OK && parts) {
                DigitGemmOut od;
                od.outd = outd;
                od.ldo = N;
                od.epA = epA;
                od.epB = epB;
                od.part_atoms = patoms;
                r = digit_gemm_plan(&p, A, B, M, N, bn, nd, katoms, katoms, 0, od, status);
                if (r == NOF_OK) r = digit_gemm_run(p, 0);
                if (r == NOF_OK)
                    k_check_scaled<<<nblkMN, 256>>>(C2, nullptr, outd, er, ecl, M, N, nd, tolV, dmax);
            }
        }
        cudaFree(er); cudaFree(ecl); cudaFree(outf); cudaFree(outd); cudaFree(epA); cudaFree(epB);
    }
    if (r == NOF_OK) {
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

// ---------------------------------------------------------------------------------------
// Timing of one GEMM shape and output mode on zero operands (measurement only; the tensor
// cores and copies do the same work whatever the digits are).
// ---------------------------------------------------------------------------------------
extern "C" int nof_bench_digit_gemm(int M, int N, int bn, int nd, int katoms, int chunk_atoms, int mode, int reps,
                                    double* us_per_launch) {
    const bool cold = mode & 4;     // L2 flushed before every timed launch
    const bool dynamic = mode & 8;  // tiles taken by a fetch-and-add counter
    const bool bad_bits = mode < 0 || (mode >> 4) != 0;
    mode &= 3;
    if (!us_per_launch || M <= 0 || N <= 0 || (nd != 4 && nd != 5) || !digit_bn_ok(bn, nd) || katoms <= 0 ||
        chunk_atoms <= 0 || bad_bits || mode > 2 || reps <= 0 ||
        (mode == 2 && chunk_atoms % digit_scale_part_atoms(nd)) || (mode != 0 && mode != 2 && chunk_atoms < katoms)) {
        nof_set_error("nof_bench_digit_gemm: bad arguments");
        return NOF_EINVAL;
    }
    const long long na = digit_elems(128, M, katoms, nd), nb = digit_elems(bn, N, katoms, nd);
    const int patoms = digit_scale_part_atoms(nd);
    const long long nkp = (katoms + patoms - 1) / patoms, kch = (katoms + chunk_atoms - 1) / chunk_atoms;
    const long long nout = (long long)M * N * (mode == 2 ? kch : 1);
    uint16_t *A = nullptr, *B = nullptr;
    void* out = nullptr;
    int *erow = nullptr, *ecol = nullptr, *status = nullptr, *ctr = nullptr;
    int r = NOF_OK;
    auto fail = [&](cudaError_t e, const char* w) { r = nof_cuda_fail(e, w, __FILE__, __LINE__); };
    cudaError_t e;
    if ((e = cudaMalloc(&A, 2ull * na)) != cudaSuccess) fail(e, "malloc A");
    if (r == NOF_OK && (e = cudaMalloc(&B, 2ull * nb)) != cudaSuccess) fail(e, "malloc B");
    if (r == NOF_OK && (e = cudaMalloc(&out, 8ull * nout)) != cudaSuccess) fail(e, "malloc out");
    if (r == NOF_OK && (e = cudaMalloc(&ctr, sizeof(int))) != cudaSuccess) fail(e, "malloc counter");
    if (r == NOF_OK && (e = cudaMalloc(&erow, 4ull * (M > N ? M : N) * nkp)) != cudaSuccess) fail(e, "malloc exps");
    if (r == NOF_OK && (e = cudaMalloc(&ecol, 4ull * (M > N ? M : N) * nkp)) != cudaSuccess) fail(e, "malloc exps");
    if (r == NOF_OK && (e = cudaMalloc(&status, 4)) != cudaSuccess) fail(e, "malloc status");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (r == NOF_OK) {
        cudaMemset(A, 0, 2ull * na);
        cudaMemset(B, 0, 2ull * nb);
        cudaMemset(erow, 0, 4ull * (M > N ? M : N) * nkp);
        cudaMemset(ecol, 0, 4ull * (M > N ? M : N) * nkp);
        cudaMemset(status, 0, 4);
        cudaMemset(ctr, 0, sizeof(int));
        DigitGemmOut o;
        o.ldo = N;
        if (dynamic) o.tile_counter = ctr;
        if (mode == 0) {  // exact int64, split-K atomics when chunked
            o.out = (long long*)out;
            o.atomic = chunk_atoms < katoms;
        } else if (mode == 1) {  // scaled double-float
            o.outf = (float2*)out;
            o.erow = erow;
            o.ecol = ecol;
        } else {  // per-part scales, FP64 partial per K chunk
            o.outd = (double*)out;
            o.chunk_stride = (long long)M * N;
            o.epA = erow;
            o.epB = ecol;
            o.part_atoms = patoms;
        }
        DigitGemmPlan p;
        r = digit_gemm_plan(&p, A, B, M, N, bn, nd, katoms, chunk_atoms, 0, o, status);
        if (r == NOF_OK) r = digit_gemm_run(p, 0);  // warm-up
        float ms = 0.f;
        if (r == NOF_OK) {
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            if (cold) {  // each launch timed alone after a write larger than L2
                for (int i = 0; i < reps && r == NOF_OK; ++i) {
                    r = l2_flush(0);
                    cudaEventRecord(e0, 0);
                    if (r == NOF_OK) r = digit_gemm_run(p, 0);
                    cudaEventRecord(e1, 0);
                    if (r == NOF_OK && (e = cudaEventSynchronize(e1)) != cudaSuccess) fail(e, "event sync");
                    float t = 0.f;
                    if (r == NOF_OK) cudaEventElapsedTime(&t, e0, e1);
                    ms += t;
                }
            } else {
                cudaEventRecord(e0, 0);
                for (int i = 0; i < reps && r == NOF_OK; ++i) r = digit_gemm_run(p, 0);
                cudaEventRecord(e1, 0);
                if ((e = cudaEventSynchronize(e1)) != cudaSuccess) fail(e, "event sync");
                if (r == NOF_OK) cudaEventElapsedTime(&ms, e0, e1);
            }
        }
        if (r == NOF_OK) {
            *us_per_launch = 1000.0 * ms / reps;
            int hs = 0;
            if ((e = cudaMemcpy(&hs, status, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) fail(e, "copy status");
            else if (hs & NOF_DEV_TIMEOUT) {
                nof_set_error("digit GEMM benchmark: a bounded wait timed out");
                r = NOF_ETIMEOUT;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(A); cudaFree(B); cudaFree(out); cudaFree(erow); cudaFree(ecol); cudaFree(status); cudaFree(ctr);
    return r;
}

// ---------------------------------------------------------------------------------------
// Failure detection: a launch whose producer issues no copies, so that the MMA warp's wait for
// its first stage, the producer's wait for a free slot and the epilogue's wait for an
// accumulator all run out; every wait is bounded by `limit_ms`, after which the kernel sets
// NOF_DEV_TIMEOUT and returns (nothing was issued, so nothing is in flight).
// ---------------------------------------------------------------------------------------
extern "C" int nof_selftest_digit_gemm_timeout(int M, int N, int bn, int nd, int katoms, double limit_ms,
                                               double* elapsed_ms) {
    if (!elapsed_ms || M <= 0 || N <= 0 || (nd != 4 && nd != 5) || !digit_bn_ok(bn, nd) || katoms <= 0 ||
        !(limit_ms > 0.0) || limit_ms > 1000.0) {
        nof_set_error("nof_selftest_digit_gemm_timeout: bad arguments (limit 0 < limit_ms <= 1000)");
        return NOF_EINVAL;
    }
    const long long na = digit_elems(128, M, katoms, nd), nb = digit_elems(bn, N, katoms, nd);
    uint16_t *A = nullptr, *B = nullptr;
    long long* C1 = nullptr;
    int* status = nullptr;
    int r = NOF_OK;
    auto fail = [&](cudaError_t e, const char* w) { r = nof_cuda_fail(e, w, __FILE__, __LINE__); };
    cudaError_t e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaMalloc(&A, 2ull * na)) != cudaSuccess) fail(e, "malloc A");
    if (r == NOF_OK && (e = cudaMalloc(&B, 2ull * nb)) != cudaSuccess) fail(e, "malloc B");
    if (r == NOF_OK && (e = cudaMalloc(&C1, 8ull * M * N)) != cudaSuccess) fail(e, "malloc C");
    if (r == NOF_OK && (e = cudaMalloc(&status, 4)) != cudaSuccess) fail(e, "malloc status");
    if (r == NOF_OK) {
        cudaMemset(A, 0, 2ull * na);
        cudaMemset(B, 0, 2ull * nb);
        cudaMemset(status, 0, 4);
        DigitGemmOut o;
        o.out = C1;
        o.ldo = N;
        DigitGemmPlan p;
        r = digit_gemm_plan(&p, A, B, M, N, bn, nd, katoms, katoms, 0, o, status);
        if (r == NOF_OK) {
            p.g.timeout_ns = (unsigned long long)(limit_ms * 1e6);
            p.g.no_copies = 1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            cudaEventRecord(e0, 0);
            r = digit_gemm_run(p, 0);
            cudaEventRecord(e1, 0);
            if (r == NOF_OK && (e = cudaEventSynchronize(e1)) != cudaSuccess) fail(e, "event sync");
            float ms = 0.f;
            if (r == NOF_OK) cudaEventElapsedTime(&ms, e0, e1);
            *elapsed_ms = ms;
        }
    }
    if (r == NOF_OK) {
        int hs = 0;
        if ((e = cudaMemcpy(&hs, status, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) fail(e, "copy status");
        else if (hs & NOF_DEV_TIMEOUT) {
            nof_set_error("digit GEMM: a bounded wait timed out (producer issued no copies)");
            r = NOF_ETIMEOUT;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(A); cudaFree(B); cudaFree(C1); cudaFree(status);
    return r;
}
