// rid_batch.cuh -- device-side description of a batch of restrained-MD label
// jobs run by the persistent kernel k_label_fused.
#pragma once

#include "rid_internal.cuh"

// One label job: a chain (its SysDev) and R restrained runs.  All arrays are
// device memory owned by the batch pool.
struct FusedJob {
    SysDev S;
    float4* x;            // [R][N] positions
    float4* v;            // [R][N] velocities
    float4* f;            // [R][N] total force at x (valid between launches)
    const double* s0;     // [R][C]
    const double* kappa;  // [R][C]
    double* sum;          // [R][C] FP64 running sums of d = wrap(s - s0)
    double* sum2;         // [R][C]
    double* bsum;         // [R][C][B] block sums
    double* mf;           // [R][C] outputs, written when the last step is done
    double* se;
    double* sd;
    int* flags;           // [R] non-finite force or velocity
    int R, B;
    long long n_steps, n_equil, K;   // K = n_steps - n_equil samples
    long long t0, t1;     // this launch runs steps [t0, t1) (t counted from the job's first step)
    uint32_t step0;       // Philox step index of t = 0
    int init;             // t0 == 0: draw / take velocities and evaluate the force at x0 first
    int mb;               // initial velocities from the Maxwell-Boltzmann draw
};

// A unit of work: one run of one job.  Items are taken in array order by the
// persistent CTAs (the host sorts them by decreasing cost).
struct FusedItem {
    int job, run;
};

struct FusedArgs {
    const FusedJob* jobs;
    const FusedItem* items;
    int n_items;
    int* next;            // work counter, zero at launch
};

// Dynamic shared memory of k_label_fused for a chain of N beads and C CVs.
size_t rid_label_fused_smem(int N, int C, int threads);
// Launch on `s` with `threads` per CTA (128, 256 or 512) and `grid` CTAs;
// smem from rid_label_fused_smem over the largest job of the batch.
// cluster > 1: every run by a thread-block cluster of that many CTAs (at most
// 8; grid a multiple of it), each forming the forces of its slice of beads.
cudaError_t rid_launch_label_fused(const FusedArgs& A, int threads, int grid, size_t smem, cudaStream_t s,
                                   int cluster = 1);
// CTAs of k_label_fused resident per SM for a block size and shared memory size.
int rid_label_fused_occupancy(int threads, size_t smem);

// Generic gather/scatter between caller arrays, staging and the pool: one CTA
// per descriptor.  kind 0: xyz float -> float4 (w = 0); 1: float4 -> xyz
// float; 2: copy doubles; 3: copy 32-bit words; 4: zero 32-bit words (src unused).
struct CopyDesc {
    const void* src;
    void* dst;
    long long n;   // elements (beads for kinds 0/1)
    int kind;
};
void rid_launch_copy_descs(const CopyDesc* descs, int n, cudaStream_t s);
