// Exact BF16 digit-plane GEMM on tcgen05 (see digit_gemm.cu for the number format).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

// Tile widths along N the kernel supports: 16, 32, 48, 64, 80, 96 (the epilogue splits BN >= 32
// into two column halves, read from TMEM in chunks of 8 columns). The TMEM accumulators (nd levels
// x BN columns per set) take two sets when 2 nd BN <= 512 columns (the drain of one set overlaps
// the MMAs into the other) and one set otherwise (5 digits with BN >= 64, 4 digits with BN >= 80).
// Wider tiles stream fewer operand bytes per multiply-add: a K atom of a tile brings 128 + BN
// rows of digits into shared memory for 128 x BN outputs.
constexpr int kDigitBN[6] = {16, 32, 48, 64, 80, 96};
inline bool digit_bn_ok(int BN, int nd) {
    return (BN == 16 || BN == 32 || BN == 48 || BN == 64 || BN == 80 || BN == 96) && nd * BN <= 512;
}
inline int digit_nbuf(int BN, int nd) { return 2 * nd * BN <= 512 ? 2 : 1; }

struct DigitGemmArgs {
    int nd;            // digits per element (4 or 5): nd (nd + 1) / 2 plane products per K atom
    int M;             // valid rows of A (rows of the output)
    int BN;            // tile width along N (kDigitBN); B is stored in tiles of BN rows
    int tiles_n;       // N tiles
    int Nvalid;        // output columns written (<= tiles_n * BN)
    int katoms;        // K atoms (16 each) per split-K chunk; the last chunk may be shorter
    int katoms_total;  // K atoms of the operands (storage stride)
    int apart;         // atoms per accumulation (even; <= digit_part_atoms_max(nd): the leading levels'
                       // FP32 partial sums stay integers below 2^24); parts are summed in the epilogue
    int tmem_cols;     // TMEM columns allocated (power of two >= nbuf * 4 * BN)
    long long* out;    // int64 fixed-point output, row-major with leading dimension ldo
    long long ldo;
    int atomic;        // 1: atomicAdd (split-K partials), 0: store
    // scaled output: when outf != nullptr the result 2^{erow[m] + ecol[n] - 40} V is stored as a
    // double-float (float2: hi, lo) at outf[m * ldo + n] instead of the int64 V
    float2* outf;
    int isum;          // scaled output summed over the parts as int64 V (set when |V| < 2^63 is certain)
    int staged;        // scaled output of single-part tiles written through a shared-memory tile (rows
                       // stored with consecutive lanes along a row) instead of lane by lane
    const int* erow;
    const int* ecol;
    // per-part scales: when epA != nullptr the value of part gp (atoms [gp apart, (gp+1) apart)
    // of K) is 2^{epA[gp * M + m] + epB[gp * Nvalid + n] - 40} V_part, summed as double-floats
    // (each operand row carries its own scale on each part of K)
    const int* epA;
    const int* epB;
    // double output: when outd != nullptr the (scaled) result is added (atomic) or stored as FP64,
    // at outd + kc * chunk_stride for K chunk kc when chunk_stride > 0 (partials summed later)
    double* outd;
    long long chunk_stride;
    // optional maxima of |value| (scaled output only; float bits, atomicMax, caller zeroes):
    // colmax[(m / group_rows) * Nvalid + n] over the rows of a group of group_rows consecutive rows
    unsigned* colmax;
    int group_rows;
    int* status;       // device status word (NOF_DEV_TIMEOUT on a timed-out wait)
    unsigned long long timeout_ns;  // limit of every mbarrier wait (%globaltimer ns; 4 s by default)
    int no_copies;     // failure-detection test only: the producer issues no copies, so waits run out
    int stages;        // shared-memory ring slots (each 2 K atoms of A and B, nd planes)
    int nbuf;          // TMEM accumulator sets
    int tiles_m;       // 128-row blocks
    int kchunks;       // K chunks (split-K); tile order: N tile fastest, then row block, then chunk
    // dynamic tiles: after tile blockIdx.x each CTA takes its next tile by a fetch-and-add on
    // *tctr (zero before the first launch; every launch leaves it at zero); nullptr: tiles
    // round-robin over the CTAs
    int* tctr;
};

// Digit-plane storage ("tile-major, 32-byte swizzled" layout). An operand with R rows is cut
// into tiles of RT rows (RT = 128 for the M side, RT = BN for the N side; R padded to a multiple
// of RT with zero rows) and K atoms of 16. Tile rt, atom t, plane i (of nd) is one contiguous
// block of RT x 16 BF16 in the K-major layout the tensor core reads with 32-byte swizzling: row r
// at r * 32 bytes, its two 16-byte halves swapped when bit 2 of r is set (bit 4 of the byte
// address XOR bit 7). Four rows then fill all 32 banks, so the MMA reads its operands without
// bank conflicts. The two atoms and nd planes of one pipeline stage are one contiguous
// RT * 64 nd-byte block, copied to shared memory as is.
__host__ __device__ __forceinline__ long long digit_offset(int RT, int katoms, long long row, long long k,
                                                           int plane, int nd) {
    // 32-bit index arithmetic (rows and K stay below 2^31; 64-bit division is emulated)
    const unsigned ur = (unsigned)row, uk = (unsigned)k;
    unsigned tile, r;
    if ((RT & (RT - 1)) == 0) {  // power-of-two tiles (128, 16, 32, 64): shifts
#ifdef __CUDA_ARCH__
        const int sh = __ffs(RT) - 1;
#else
        const int sh = __builtin_ctz((unsigned)RT);
#endif
        tile = ur >> sh;
        r = ur & (unsigned)(RT - 1);
    } else {
        tile = ur / (unsigned)RT;
        r = ur - tile * (unsigned)RT;
    }
    const unsigned t = uk >> 4, kk = uk & 15u;
    const long long block = (((long long)tile * katoms + t) * nd + plane) * (long long)(RT * 16);
    return block + (long long)(r * 16 + ((((kk >> 3) ^ (r >> 2)) & 1u) << 3) + (kk & 7));
}
// elements of a digit tensor with R rows (padded to RT), katoms atoms and nd planes
__host__ __device__ __forceinline__ long long digit_elems(int RT, long long R, int katoms, int nd) {
    return (R + RT - 1) / RT * RT * (long long)katoms * 16 * nd;
}

// Where a GEMM writes (one of out / outf / outd) and how its parts are scaled.
struct DigitGemmOut {
    long long* out = nullptr;  // int64 V
    float2* outf = nullptr;    // scaled double-float
    double* outd = nullptr;    // FP64 (with per-part scales)
    long long chunk_stride = 0;  // > 0: FP64 partial of K chunk kc at outd + kc * chunk_stride
    long long ldo = 0;
    bool atomic = false;
    const int* erow = nullptr;
    const int* ecol = nullptr;
    const int* epA = nullptr;  // per-part scales [parts][M] and [parts][Nvalid]; parts of part_atoms
    const int* epB = nullptr;
    unsigned* colmax = nullptr;
    int group_rows = 1;
    int part_atoms = 0;  // per-part scales: K atoms per part (digit_scale_part_atoms; a chunk is whole parts)
    int* tile_counter = nullptr;  // dynamic tiles (DigitGemmArgs::tctr); one counter per plan in use
};
// Digit contract. Every digit lies in [-128, 128] except the leading one, which lies in
// [-digit_top(nd), digit_top(nd)]: with 5 digits the row scale leaves one bit of headroom so that
// the leading digit is bounded like the others (39 significant bits), with 4 digits it does not
// (32 bits, |d_0| <= 256). digit_headroom(nd) is that extra bit of the scale exponent.
__host__ __device__ inline int digit_headroom(int nd) { return nd == 5 ? 1 : 0; }
__host__ __device__ inline int digit_top(int nd) { return nd == 5 ? 128 : 256; }
// Longest accumulation in K atoms: the leading levels 0 .. nd - 3 must stay exact, i.e. below 2^24.
// Level 2 (5 digits) receives at most 3 128^2 per K element: 341 elements, 20 atoms (even). Level 1
// (4 digits) receives at most 2 256 128: 256 elements, 16 atoms.
inline int digit_part_atoms_max(int nd) { return nd == 5 ? 20 : 16; }
// K atoms of one part of the per-part scales (the Lagrangian contraction, whose K runs over every
// aux index): longer parts mean fewer accumulator drains (each part is drained and scaled on its
// own), shorter ones finer scales; 5 digits take the longest exact part, 4 digits, which have
// less precision to spare, the finer scales.
inline int digit_scale_part_atoms(int nd) { return nd == 5 ? 20 : 8; }

// A launch plan (pointers and shapes fixed at set-up).
struct DigitGemmPlan {
    const uint16_t* A;
    const uint16_t* B;
    DigitGemmArgs g;
    dim3 grid;
    size_t smem;
};

// Plan C = A B^T for A (M x 16 katoms_total, nd digit planes, row tiles of 128) and B (tiles of
// BN rows), split-K in chunks of chunk_atoms; stages = 0 picks the deepest ring that fits.
int digit_gemm_plan(DigitGemmPlan* plan, const uint16_t* A, const uint16_t* B, int M, int Nvalid, int BN,
                    int nd, int katoms_total, int chunk_atoms, int stages, const DigitGemmOut& out,
                    int* status);
int digit_gemm_run(const DigitGemmPlan& plan, cudaStream_t st);
int digit_gemm_max_stages(int BN, int nd, bool staged = false);

// Autotuner: times every candidate (one warm-up launch, then the best of three timed with CUDA
// events on `st`; with `cold`, each timed launch follows an L2 flush, as for a GEMM whose operands
// were last touched long before) and returns the index of the fastest. Results are remembered per `key` for the
// life of the process, so equal shapes are timed once.
struct DigitTuneKey {
    int kind, M, Nvalid, katoms_total, extra;
};
int digit_gemm_pick(const DigitTuneKey& key, const DigitGemmPlan* cands, int ncand, cudaStream_t st, int* best,
                    bool cold = false);
// Write a buffer twice the size of L2 on `st` (timing of launches whose operands come from HBM).
int l2_flush(cudaStream_t st);
