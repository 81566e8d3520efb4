// Exact BF16 digit-plane GEMM on tcgen05 (see digit_gemm.cu for the number format).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

struct DigitGemmArgs {
    int M;          // valid rows of A (rows of the output)
    int N;          // padded N (multiple of 16, <= 128); B has N rows
    int Nvalid;     // columns written
    int katoms;     // K atoms (16 each) accumulated per CTA (<= 10: exact for K <= 160)
    int tmem_cols;  // TMEM columns allocated (power of two >= 4 N)
    long long* out; // int64 fixed-point output, row-major with leading dimension ldo
    long long ldo;
    int atomic;     // 1: atomicAdd (split-K partials), 0: store
    int* status;    // device status word (NOF_DEV_TIMEOUT on a timed-out wait)
};

// A launch with its tensor maps encoded once (they depend only on buffer addresses and sizes).
struct DigitGemmPlan {
    CUtensorMap ma, mb;
    DigitGemmArgs g;
    dim3 grid;
    size_t smem;
};

size_t digit_gemm_smem(int N);
int digit_gemm_plan(DigitGemmPlan* plan, const uint16_t* A, int rowsA, const uint16_t* B, int N,
                    int katoms_total, int katoms, int M, int Nvalid, long long* out, long long ldo,
                    bool atomic, int* status);
int digit_gemm_run(const DigitGemmPlan& plan, cudaStream_t st);
int digit_gemm(const uint16_t* A, int rowsA, const uint16_t* B, int N, int katoms_total, int katoms,
               int M, int Nvalid, long long* out, long long ldo, bool atomic, int* status,
               cudaStream_t st);
