// rid_internal.cuh -- device-side data layout and shared device helpers of
// librid.  Included by every .cu file of the library.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "rid.h"

// A named NVTX range over the lifetime of the object: each public call and
// each server tick shows as one range in a profiler that records NVTX (a
// no-op when none is attached).
struct NvtxScope {
    explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope&) = delete;
    NvtxScope& operator=(const NvtxScope&) = delete;
};

#define RID_MAX_LAYERS 8
#define RID_MAX_MODELS 16
#define RID_MAX_CV 128
#define RID_MAX_BEADS 4096
#define RID_MAX_WIDTH 512
#define RID_MAX_BLOCKS 256
#define RID_BONDED_SMEM_MAX 1024

// --------------------------------------------------------------------------
// Parameters of one bead-chain system, passed by value to kernels.
struct SysDev {
    int N, C, output_freq;
    float inv_mass, half_dt, c1, c2, sd_mb;   // c1 = e^{-gamma dt}, c2 = sqrt((1-c1^2) kT/m)
    float kb, r0, ka, th0;
    float lj_eps24, lj_eps4, sig2, rc2, urc; // urc: U_LJ(rc) shift
    uint32_t key0, key1;
    const float* dih;        // [N-3][6]: k_1, k_2, k_3, delta_1, delta_2, delta_3
    const int4* cv;          // [C] bead quadruples (z < 0: the distance between x and y)
    const int* acv_off;      // [N+1] CSR offsets: CV slots touching each bead
    const int2* acv;         // (cv index, slot 0..3), ordered by cv index
};

// Ensemble weights on the device, FP32 (plain path).
struct EnsDev {
    int M, D, L, H, resnet;
    int aslices;             // member values come as [M][aslices][W] partial sums
    float e0, e1;
    const float* W;          // per model, per layer: row-major [H][fin]
    const float* WT;         // per model, per layer: row-major [fin][H]
    const float* b;          // [M][L][H]
    const float* wout;       // [M][H]
    const float* bout;       // [M]
    long long wstride;       // floats per model in W / WT
    long long loff[RID_MAX_LAYERS];  // offset of layer l within a model
    const int* cvdist;       // [C] 1 for a distance CV (input (s, 0)), or NULL when all are torsions
};

// Resident walker state (capacity W walkers).
struct StateDev {
    int W;
    float4* x;      // [W][N] positions (w unused)
    float4* v;      // [W][N] velocities
    float4* f;      // [W][N] total force of the last evaluation
    float4* fff;    // [W][N] force-field part of the current evaluation
    float* s;       // [W][C] CVs
    float4* J;      // [W][C][4] dCV/dx for the four beads
    float* u;       // [W][D] MLP input (cos, sin) FP32
    float* gradA;   // [M][W][C] member CV gradients
    float* Aval;    // [M][W] member values
    float* eps;     // [W] model deviation of the current evaluation
    float* hs;      // MLP activation scratch
    double* eff;    // [W] force-field energy (energy mode)
    int* flags;     // [W] non-finite flags
    const uint32_t* stepbase;   // device base added to the Philox step index (graph replay), or NULL
};

// Label (restrained MD) accumulators.
struct LabelDev {
    const double* s0;     // [W][C]
    const double* kappa;  // [W][C]
    double* sum;          // [W][C]
    double* sum2;         // [W][C]
    double* bsum;         // [W][C][B]
    int B;
    long long n_equil, K; // K = samples = n_steps - n_equil
};

// --------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 products
// on words 0 and 2, mixed with words 1, 3 and the key, key bumped by the Weyl
// constants after each round.
__device__ __forceinline__ uint4 rid_philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// -2 ln u for u = (x + 1/2) 2^-32, accurate in FP32 over the whole range:
// for x >= 2^31 it works from 1 - u = (~x + 1/2) 2^-32 through log1p.
__device__ __forceinline__ float rid_m2logu(uint32_t x) {
    if (x < 0x80000000u) {
        const float u = fmaf(__uint2float_rn(x), 0x1p-32f, 0x1p-33f);
        return -2.0f * logf(u);
    }
    const float om = fmaf(__uint2float_rn(~x), 0x1p-32f, 0x1p-33f);
    return -2.0f * log1pf(-om);
}

// Three standard normals from one counter: Box-Muller on words (0,1) and (2,3).
__device__ __forceinline__ float3 rid_normals3(uint4 w) {
    const float r0 = sqrtf(rid_m2logu(w.x));
    const float r1 = sqrtf(rid_m2logu(w.z));
    float s0, c0, s1, c1;
    sincospif(fmaf(__uint2float_rn(w.y), 0x1p-31f, 0x1p-32f), &s0, &c0);
    sincospif(fmaf(__uint2float_rn(w.w), 0x1p-31f, 0x1p-32f), &s1, &c1);
    (void)s1;
    return make_float3(r0 * c0, r0 * s0, r1 * c1);
}

// --------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Torsion angle (IUPAC sign, [-pi, pi)) and optionally its gradient w.r.t.
// the four points.  With F = p0-p1, G = p1-p2, H = p3-p2, A = F x G and
// B = H x G:  phi = atan2(-|G| F.B, A.B), and (Blondel & Karplus 1996)
//   dphi/dp0 = -|G|/A^2 A,  dphi/dp3 = |G|/B^2 B,
//   dphi/dp1 = (|G|/A^2 + F.G/(A^2|G|)) A - H.G/(B^2|G|) B,
//   dphi/dp2 = (H.G/(B^2|G|) - |G|/B^2) B - F.G/(A^2|G|) A.
__device__ __forceinline__ float rid_torsion(float3 p0, float3 p1, float3 p2, float3 p3, float3* g) {
    const float3 F = p0 - p1, G = p1 - p2, H = p3 - p2;
    const float3 A = cross3(F, G), B = cross3(H, G);
    const float lG = sqrtf(dot3(G, G));
    float phi = atan2f(-lG * dot3(F, B), dot3(A, B));
    if (phi >= 3.14159265358979f) phi -= 6.28318530717959f;
    if (g) {
        const float A2 = dot3(A, A), B2 = dot3(B, B);
        const float ia = lG / A2, ib = lG / B2;
        const float ca = dot3(F, G) / (A2 * lG), cb = dot3(H, G) / (B2 * lG);
        g[0] = (-ia) * A;
        g[3] = ib * B;
        g[1] = (ia + ca) * A - cb * B;
        g[2] = (cb - ib) * B - ca * A;
    }
    return phi;
}

// One CV of a system (Sec. "CV selection"): q = (a, b, c, d) is the torsion
// of four beads, or, when q.z < 0, the distance |x_b - x_a| (not periodic).
// Returns s and its gradient on the CV's four slots (a distance fills slots
// 0 and 1 with -(x_b - x_a)/s and +(x_b - x_a)/s, slots 2 and 3 with zero).
__device__ __forceinline__ bool rid_cv_is_distance(int4 q) { return q.z < 0; }
template <typename X>
__device__ __forceinline__ float rid_cv(int4 q, const X* xs, float3* g) {
    if (rid_cv_is_distance(q)) {
        const float3 r = f3(xs[q.y]) - f3(xs[q.x]);
        const float d = sqrtf(dot3(r, r));
        const float id = 1.0f / d;
        g[1] = id * r;
        g[0] = make_float3(-g[1].x, -g[1].y, -g[1].z);
        g[2] = g[3] = make_float3(0.f, 0.f, 0.f);
        return d;
    }
    return rid_torsion(f3(xs[q.x]), f3(xs[q.y]), f3(xs[q.z]), f3(xs[q.w]), g);
}
// MLP input pair of a CV: (cos s, sin s) for a torsion, (s, 0) for a distance.
__device__ __forceinline__ void rid_cv_input(int4 q, float s, float& u0, float& u1) {
    if (rid_cv_is_distance(q)) {
        u0 = s;
        u1 = 0.0f;
    } else {
        sincosf(s, &u1, &u0);
    }
}

// wrap onto [-pi, pi): d - 2 pi floor(d / 2 pi + 1/2)
__device__ __forceinline__ float rid_wrapf(float d) {
    return d - 6.28318530717959f * floorf(d * 0.159154943091895f + 0.5f);
}
__device__ __forceinline__ double rid_wrapd(double d) {
    return d - 6.283185307179586 * floor(d * 0.15915494309189535 + 0.5);
}
// Restraint offset of a CV from its centre: wrapped for a torsion, plain for
// a distance.
__device__ __forceinline__ double rid_cv_offset(int4 q, double s, double s0) {
    return rid_cv_is_distance(q) ? s - s0 : rid_wrapd(s - s0);
}

// --------------------------------------------------------------------------
// cudaFuncSetAttribute acts on the current device only: a launcher that opts
// a kernel into more shared memory asks this first, and it answers true once
// per device (one bit of `done` per device ordinal).
inline bool rid_first_on_device(unsigned long long& done) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return true;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done & bit) return false;
    done |= bit;
    return true;
}

// --------------------------------------------------------------------------
// Host-side kernel launchers (defined in the .cu files).
void rid_launch_pack(const float* src, float4* dst, long long n, cudaStream_t st);
void rid_launch_unpack(const float4* src, float* dst, long long n, cudaStream_t st);
void rid_launch_mb(const SysDev& S, StateDev st, int W, uint32_t step0, cudaStream_t s);
void rid_launch_pair_mask(const SysDev& S, StateDev st, int W, uint32_t* mask, cudaStream_t s);
int rid_ff_smem_bytes(int N);
size_t rid_label_cons_smem(int N, int C);
// CV kinds of an MCMC run: dist [C] (1: a distance CV, not periodic, moved and
// binned inside [lo, hi]; NULL: every CV a torsion), lo / hi [C].
struct McCvDev {
    const int* dist = nullptr;
    const float* lo = nullptr;
    const float* hi = nullptr;
};
void rid_launch_mc_features(const float* s, float* U, long long n, int C, const McCvDev& cvk, cudaStream_t st);
void rid_launch_mc_propose(const float* s, float* sp, float* U, int W, int C, uint32_t step, float step_size,
                           uint32_t k0, uint32_t k1, const McCvDev& cvk, cudaStream_t st);
// Device side of a path projection (n_nodes = 0: off).
struct McPathDev {
    int n_nodes = 0, n_cv = 0;
    const int* cv = nullptr;               // [n_cv]
    const float* nodes = nullptr;          // [n_nodes][n_cv]
    float lambda = 0.0f, z_lo = 0.0f, z_hi = 0.0f;
    unsigned long long* hist = nullptr;    // [bins][bins]
};
// Checks the ranges of the distance CVs of an MCMC run (RID_OK or RID_ERR_ARG).
int rid_mc_range_check(int C, const int32_t* dist, const double* lo, const double* hi);
// Checks a path projection's host arguments against C CVs (RID_OK or RID_ERR_ARG).
int rid_mc_path_check(int n_nodes, int n_cv, int C, const int32_t* cv, const float* nodes, double lambda,
                      double z_lo, double z_hi);
void rid_launch_mc_accept_values(const float* aval, int na, int M, int W, int C, float* s, const float* sp, float* A,
                                 uint32_t step, float kT, uint32_t k0, uint32_t k1, int init, int count, int bins,
                                 int pi, int pj, unsigned long long* hist1, unsigned long long* hist2,
                                 unsigned long long* nacc, const McPathDev& path, const McCvDev& cvk,
                                 cudaStream_t st);
void rid_launch_mc_pmf(const unsigned long long* hist, int rows, int n, double kT, double* pmf, cudaStream_t st);
cudaError_t rid_launch_label_cons(const SysDev& S, int R, int C, int B, long long n_steps, long long n_equil,
                                  uint32_t step0, float kT, const float4* x0, const float4* v0, const int2* pairs,
                                  const float* d0, double* bsum, double* mf, double* se, double* sd, float4* x_out,
                                  float4* v_out, int* bad, cudaStream_t st);
void rid_launch_ff(const SysDev& S, StateDev st, int W, bool energy, cudaStream_t s, int threads = 0);
int rid_ff_default_threads(int N);

// Arguments of the fused finish / B-A-O-A / CV kernel.
struct HeadArgs {
    SysDev S;
    StateDev st;
    EnsDev E;
    LabelDev lab;
    int W, mode;
    bool fin, kick, energy;
    int integ;                 // 0 none, 1 CVs at current positions, 2 B-A-O-A then CVs
    long long t_fin;           // local index of the step being finished
    int slot;                  // trace slot of that step, -1 for none
    float* cv_out;
    float* eps_out;
    double* energy_out;
    long long T;
    uint32_t step;             // Philox step of the opened step
    bool no_split;             // one CTA per walker whatever W (a server's jobs: measured better under
                               // concurrency than clusters per walker)
};
void rid_launch_head(const HeadArgs& a, cudaStream_t s);
// Every step of an exploration call in one persistent launch (k_explore_small):
// shared memory it needs, 0 when the shape is not eligible.
size_t rid_explore_small_smem(const SysDev& S, const EnsDev& E);
cudaError_t rid_launch_explore_small(const SysDev& S, StateDev st, const EnsDev& E, int W, long long n_steps,
                                     uint32_t step0, float* cv_out, float* eps_out, long long T, cudaStream_t s);
void rid_launch_add_u32(uint32_t* p, uint32_t d, cudaStream_t s);
void rid_launch_label_final(const LabelDev& lab, int W, int C, double* mf, double* se, double* sd,
                            cudaStream_t s);
void rid_launch_philox(long long n, const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* words,
                       float* normals, cudaStream_t s);
void rid_launch_mlp_fp32(const EnsDev& E, StateDev st, int W, int C, cudaStream_t s);
size_t rid_mlp_fp32_scratch_floats(int W, int M, int L, int H);
// Set the calling thread's rid_last_error message; returns code.
int rid_fail(int code, const char* fmt, ...);
// Device description and device ordinal of a system (defined with rid_system).
const SysDev* rid_sys_dev(const rid_system* sys);
int rid_sys_device(const rid_system* sys);
// Resident-walker operations used by the request loop (all enqueue on st).
//   load: W walkers from host arrays (v0 NULL: Maxwell-Boltzmann), force at x0,
//     Philox step base = step0.
//   graph_advance: capture n_steps biased steps (n_steps a multiple of the
//     output frequency) with device traces dcv [W][T][C], deps [W][T] as a
//     graph whose Philox step index is read from the device base, which the
//     graph advances by n_steps at its end; the graph can be replayed.
//   advance: the same steps launched directly (for a remainder chunk).
//   read_async: unpack x, v (either may be NULL) into device xyz arrays.
//   flags: whether any walker went non-finite since the load (synchronises st).
int rid_sys_load(rid_system* sys, int W, const float* x0, const float* v0, uint64_t step0, cudaStream_t st);
// while on, the system's kernels run without their tuners (see rid_system::serving)
void rid_sys_serving(rid_system* sys, bool on);
int rid_sys_graph_advance(rid_system* sys, int64_t n_steps, float* dcv, float* deps, cudaStream_t st,
                          cudaGraphExec_t* out);
int rid_sys_advance(rid_system* sys, int64_t n_steps, float* dcv, float* deps, cudaStream_t st);
int rid_sys_read_async(rid_system* sys, float* dx, float* dv, cudaStream_t st);
int rid_sys_flags(rid_system* sys, cudaStream_t st, bool* any_bad);
// Device bytes a system holds for W walkers with its current ensemble.
size_t rid_sys_footprint(const rid_system* sys, int W);
