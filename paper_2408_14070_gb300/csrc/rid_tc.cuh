// rid_tc.cuh -- arguments of the tcgen05 BF16 ensemble-MLP kernel.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "rid_internal.cuh"

#define TC_MAX_STAGES 8

// Weight images: for every member, GEMM g (forward layers 0..L-1, then
// backward layers L-1..0), K-chunk c and cluster rank q, the B-operand slice
// rows [q N_g/CS, (q+1) N_g/CS) x columns [c ck, (c+1) ck) stored exactly as
// the canonical no-swizzle K-major shared-memory layout: 8-row x 16-byte core
// matrices, k-block-major ([ck/8][rows/8][8][8] BF16).  Offsets are in rows of
// 128 bytes (the tensor map's inner box).
struct TcArgs {
    int W, C, D, Dp, L, H, M, CS, ck, stages, Kmax, ntiles, tmem_cols;
    unsigned stage_bytes;
    const float* u;          // [W][D] MLP input (cos, sin), FP32
    const float* bias;       // [M][L][H]
    const float* wout;       // [M][H]
    const float* bout;       // [M]
    __nv_bfloat16* tsave;    // [M][ntiles][L][128][H] tanh(z_l), BF16
    float* gradA;            // [M][W][C]
    float* Apart;            // [M][CS][W] member value, per column slice
    int* err;                // error word (bounded-wait expiry codes)
    long long member_rows;   // 128-byte rows per member image
    long long grow[2 * RID_MAX_LAYERS];   // first row of GEMM g within a member image
    int gN[2 * RID_MAX_LAYERS], gK[2 * RID_MAX_LAYERS];
};

size_t rid_mlp_tc_smem_bytes(const TcArgs& P);
cudaError_t rid_launch_mlp_tc(const TcArgs& P, const CUtensorMap& big, const CUtensorMap& small, cudaStream_t s);
