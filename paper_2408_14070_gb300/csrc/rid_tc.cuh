// rid_tc.cuh -- arguments of the tcgen05 BF16 ensemble-MLP kernel.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "rid_internal.cuh"

#define TC_MAX_STAGES 8
#define TC_MAX_KCHUNKS 8   // 128-byte K-chunks of the widest GEMM (K <= 512 BF16)
#define TC_MAX_QSLICES 32  // 16-column slices of the widest hidden layer (512)

// Weight image, per member: for GEMM g (forward layers 0..L-1, then backward
// layers L-1..0) and K-chunk c (128 bytes of K: 64 BF16 or 128 FP8 e4m3
// columns), the B operand rows [0, N_g) x that column range as rows of 128
// bytes in the 128-byte swizzled layout (16-byte chunk j of row n at position
// j ^ (n mod 8)), zero padded beyond K_g.  Offsets are counted in those
// 128-byte rows.  FP8 matrices hold W / s with s = amax|W| / 448 per member
// and matrix.
struct TcArgs {
    int W, C, D, Dp, L, H, M;
    int stages, Kpmax, ntiles, tmem_cols, nacc, acc_cols;   // Kpmax: A-tile row bytes / 2
    unsigned stage_bytes;
    const float* u;          // [W][D] MLP input (cos, sin) or (s, 0), FP32
    const int* cvdist;       // [C] 1 for a distance CV, or NULL when all are torsions
    const float* bias;       // [M][L][H]
    const float* wout;       // [M][H]
    const float* bout;       // [M]
    __nv_bfloat16* tsave;    // [M][ntiles][L][128][H] tanh(z_l), BF16
    float* gradA;            // [M][W][C]
    float* Apart;            // [M][W] member value
    float* qsave;            // [M][ntiles][TC_MAX_QSLICES][128] partial member values per 16-column slice
    int* err;                // error word (bounded-wait expiry codes)
    long long member_rows;   // 128-byte rows per member image
    long long grow[2 * RID_MAX_LAYERS];          // first row of GEMM g within a member image
    int gN[2 * RID_MAX_LAYERS], gKp[2 * RID_MAX_LAYERS];   // N, and K padded to a 128-byte chunk
    int geb[2 * RID_MAX_LAYERS];                           // operand bytes per element: 2 BF16, 1 FP8 e4m3
    const float* wscale;     // [M][2L] weight scale of every GEMM (1 for BF16)
    int resnet;              // h_l = h_{l-1} + tanh(z_l) for l >= 1
    float* rsave;            // resnet: [M][ntiles][H/8][128][8] FP32, h_l forward, dA/dh_l backward
    int csize;               // cluster variant: CTAs splitting each GEMM's output columns (2 or 4)
    int ngemm;               // GEMMs to run: 2L (forward and input gradient) or L (forward only:
                             // member values, gradA untouched)
};

size_t rid_mlp_tc_smem_bytes(const TcArgs& P);
cudaError_t rid_launch_mlp_tc(const TcArgs& P, const CUtensorMap& big, const CUtensorMap& small, cudaStream_t s);
size_t rid_mlp_tc_wide_smem_bytes(const TcArgs& P);
cudaError_t rid_launch_mlp_tc_wide(const TcArgs& P, const CUtensorMap& big, const CUtensorMap& small, cudaStream_t s);
// Small walker counts (up to 16: NW = 16 MMA columns), BF16, forward and
// input gradient: the GEMMs transposed (outputs on the MMA's M = 128 rows,
// walkers on its N columns), each GEMM's 128-output tiles split over a cluster
// of P.csize (1..4) CTAs per member.
size_t rid_mlp_tc_small_smem_bytes(const TcArgs& P, int NW);
// epi_warps: 16, or 8 (the lean variant: half the threads, same results bit for bit)
cudaError_t rid_launch_mlp_tc_small(const TcArgs& P, const CUtensorMap& big, const CUtensorMap& small, int NW,
                                    int epi_warps, cudaStream_t s);
size_t rid_mlp_tc_cluster_smem_bytes(const TcArgs& P);
cudaError_t rid_launch_mlp_tc_cluster(const TcArgs& P, const CUtensorMap& big, const CUtensorMap& small,
                                      cudaStream_t s);
