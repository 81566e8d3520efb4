// Exact BF16 digit-plane GEMM on tcgen05 (see digit_gemm.cu for the number format).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

struct DigitGemmArgs {
    int M;          // valid rows of A (rows of the output)
    int N;          // padded N (multiple of 16, <= 128); B has N rows
    int Nvalid;     // columns written
    int katoms;     // K atoms (16 each) accumulated per tile
    int kparts;     // exact accumulations per tile: atoms [p * apart, (p + 1) * apart) go to TMEM level
    int apart;      // set p (apart <= 10 keeps every FP32 partial sum exact); parts are summed in the epilogue
    int katoms_total;  // K atoms of the whole operand (storage stride)
    int tmem_cols;  // TMEM columns allocated (power of two >= 4 N)
    long long* out; // int64 fixed-point output, row-major with leading dimension ldo
    long long ldo;
    int atomic;     // 1: atomicAdd (split-K partials), 0: store
    // scaled output: when outf != nullptr the result 2^{erow[m] + ecol[n] - 40} V is stored as a
    // double-float (float2: hi, lo) at outf[m * ldo + n] instead of the int64 V
    float2* outf;
    const int* erow;
    const int* ecol;
    int* status;    // device status word (NOF_DEV_TIMEOUT on a timed-out wait)
    int stages;     // shared-memory ring slots (each 2 K atoms of A and B, 4 planes)
    int nbuf;       // TMEM accumulator sets (2 when 8 N <= 512 columns)
    int tiles_m;    // 128-row blocks
    int kchunks;    // K chunks (split-K); tiles = tiles_m * kchunks, row block fastest
};

// Digit-plane storage ("tile-major core-matrix" layout). An operand with R rows is cut into tiles
// of RT rows (RT = 128 for the M side, RT = N for the N side; R padded to a multiple of RT with
// zero rows) and K atoms of 16. Tile rt, atom t, plane i is one contiguous block of RT x 16 BF16
// in the order the tensor core reads without swizzling: 8-row x 8-element core matrices
// (128 bytes) ordered [row group r/8][k half kk/8][row r%8][element kk%8]. The two atoms and four
// planes of one pipeline stage are therefore one contiguous RT * 256-byte block.
__host__ __device__ __forceinline__ long long digit_offset(int RT, int katoms, long long row, long long k,
                                                           int plane) {
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
    const long long block = (((long long)tile * katoms + t) * 4 + plane) * (long long)(RT * 16);
    return block + (long long)(((r >> 3) * 2 + (kk >> 3)) * 64 + (r & 7) * 8 + (kk & 7));
}
// elements of a digit tensor with R rows (padded to RT) and katoms atoms
__host__ __device__ __forceinline__ long long digit_elems(int RT, long long R, int katoms) {
    return (R + RT - 1) / RT * RT * (long long)katoms * 16 * 4;
}

// A launch plan (pointers and shapes fixed at set-up).
struct DigitGemmPlan {
    const uint16_t* A;
    const uint16_t* B;
    DigitGemmArgs g;
    dim3 grid;
    size_t smem;
};

size_t digit_gemm_smem(int N);
int digit_gemm_plan(DigitGemmPlan* plan, const uint16_t* A, const uint16_t* B, int N, int katoms_total,
                    int katoms, int M, int Nvalid, long long* out, long long ldo, bool atomic, int* status);
// Same GEMM with the scaled double-float output (value = 2^{erow[m] + ecol[n] - 40} V).
int digit_gemm_plan_scaled(DigitGemmPlan* plan, const uint16_t* A, const uint16_t* B, int N, int katoms,
                           int M, int Nvalid, float2* out, long long ldo, const int* erow, const int* ecol,
                           int* status);
int digit_gemm_run(const DigitGemmPlan& plan, cudaStream_t st);
int digit_gemm(const uint16_t* A, const uint16_t* B, int N, int katoms_total, int katoms, int M,
               int Nvalid, long long* out, long long ldo, bool atomic, int* status, cudaStream_t st);
