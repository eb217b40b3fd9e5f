// k_step.cu -- per-walker kernels of the RiD Langevin step on sm_103a.
//
// One CTA owns one walker (bead chain) for the whole evaluation: the chain's
// positions are staged once in shared memory and every force term reads them
// from there.  All sums are taken in a fixed order, so results are
// bit-reproducible run to run.
//
//   k_force_cv  : [B A O A of BAOAB] + force field (bonds, angles, dihedrals,
//                 all-pairs Lennard-Jones) + torsion CVs and their Jacobians
//   k_finish    : CV force (ensemble bias with the trust-level switch, or a
//                 harmonic restraint with FP64 label sums) chain-ruled to the
//                 beads + the closing B half-kick + trace output
#include <math.h>

#include "rid_internal.cuh"

namespace {


__global__ void k_pack(const float* __restrict__ src, float4* __restrict__ dst, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = make_float4(src[3 * i], src[3 * i + 1], src[3 * i + 2], 0.0f);
}

__global__ void k_unpack(const float4* __restrict__ src, float* __restrict__ dst, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const float4 a = src[i];
        dst[3 * i] = a.x;
        dst[3 * i + 1] = a.y;
        dst[3 * i + 2] = a.z;
    }
}

// Maxwell-Boltzmann velocities: Philox stream 1 at counter (bead, walker, step0, 1).
__global__ void k_mb(SysDev S, StateDev st, int W, uint32_t step0) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)W * S.N) return;
    const int w = (int)(idx / S.N), i = (int)(idx % S.N);
    const float3 z = rid_normals3(rid_philox(make_uint4(i, w, step0, 1u), S.key0, S.key1));
    st.v[idx] = make_float4(S.sd_mb * z.x, S.sd_mb * z.y, S.sd_mb * z.z, 0.0f);
}

// ---------------------------------------------------------------------------
// Bonded terms, gathered per bead (each term is evaluated by every bead it
// touches, which keeps the sums ordered and needs no atomics).

// Force on p from the harmonic bond p-q.
__device__ __forceinline__ float3 bond_force(const SysDev& S, float3 p, float3 q) {
    const float3 d = q - p;
    const float r = sqrtf(dot3(d, d));
    return (S.kb * (r - S.r0) / r) * d;
}

// Harmonic angle a-c-b (vertex c): forces on a, c, b.
__device__ __forceinline__ void angle_forces(const SysDev& S, float3 pa, float3 pc, float3 pb, float3& fa,
                                             float3& fc, float3& fb) {
    const float3 a = pa - pc, b = pb - pc;
    const float3 axb = cross3(a, b);
    const float cr = sqrtf(dot3(axb, axb)), dp = dot3(a, b);
    const float th = atan2f(cr, dp);
    const float dU = S.ka * (th - S.th0);
    const float ia = 1.0f / cr;
    const float3 ga = ia * ((dp / dot3(a, a)) * a - b);   // d theta / d a
    const float3 gb = ia * ((dp / dot3(b, b)) * b - a);   // d theta / d b
    fa = (-dU) * ga;
    fb = (-dU) * gb;
    fc = dU * (ga + gb);
}

// Dihedral k (beads k..k+3): -dU/dphi and the torsion gradient.
__device__ __forceinline__ float dihedral_mdU(const SysDev& S, int k, float phi) {
    const float* p = S.dih + 6 * k;
    float m = 0.0f;
#pragma unroll
    for (int n = 1; n <= 3; ++n) m = fmaf((float)n * p[n - 1], sinf((float)n * phi - p[2 + n]), m);
    return m;   // -dU/dphi = sum_n n k_n sin(n phi - delta_n)
}

__device__ __forceinline__ float dihedral_energy(const SysDev& S, int k, float phi) {
    const float* p = S.dih + 6 * k;
    float e = 0.0f;
#pragma unroll
    for (int n = 1; n <= 3; ++n) e += p[n - 1] * (1.0f + cosf((float)n * phi - p[2 + n]));
    return e;
}

__device__ float3 bonded_force_on(const SysDev& S, const float4* xs, int i) {
    const int N = S.N;
    const float3 xi = f3(xs[i]);
    float3 f = make_float3(0.f, 0.f, 0.f);
    if (i > 0) f = f + bond_force(S, xi, f3(xs[i - 1]));
    if (i + 1 < N) f = f + bond_force(S, xi, f3(xs[i + 1]));
    float3 fa, fc, fb;
    if (i + 2 < N) { angle_forces(S, xi, f3(xs[i + 1]), f3(xs[i + 2]), fa, fc, fb); f = f + fa; }
    if (i >= 1 && i + 1 < N) { angle_forces(S, f3(xs[i - 1]), xi, f3(xs[i + 1]), fa, fc, fb); f = f + fc; }
    if (i >= 2) { angle_forces(S, f3(xs[i - 2]), f3(xs[i - 1]), xi, fa, fc, fb); f = f + fb; }
    const int d0 = i - 3 > 0 ? i - 3 : 0;
    const int d1 = i < N - 4 ? i : N - 4;
    for (int k = d0; k <= d1; ++k) {
        float3 g[4];
        const float phi = rid_torsion(f3(xs[k]), f3(xs[k + 1]), f3(xs[k + 2]), f3(xs[k + 3]), g);
        const int q = i - k;   // select without a dynamic index (keeps g in registers)
        const float3 gq = q == 0 ? g[0] : (q == 1 ? g[1] : (q == 2 ? g[2] : g[3]));
        f = f + dihedral_mdU(S, k, phi) * gq;
    }
    return f;
}

// Energy of the bonded terms that start at bead i (bond i,i+1; angle i..i+2;
// dihedral i..i+3), so that every term is counted once.
__device__ double bonded_energy_from(const SysDev& S, const float4* xs, int i) {
    const int N = S.N;
    double e = 0.0;
    const float3 xi = f3(xs[i]);
    if (i + 1 < N) {
        const float3 d = f3(xs[i + 1]) - xi;
        const float dr = sqrtf(dot3(d, d)) - S.r0;
        e += 0.5 * S.kb * (double)dr * dr;
    }
    if (i + 2 < N) {
        const float3 a = xi - f3(xs[i + 1]), b = f3(xs[i + 2]) - f3(xs[i + 1]);
        const float3 axb = cross3(a, b);
        const float dth = atan2f(sqrtf(dot3(axb, axb)), dot3(a, b)) - S.th0;
        e += 0.5 * S.ka * (double)dth * dth;
    }
    if (i + 3 < N) {
        const float phi = rid_torsion(xi, f3(xs[i + 1]), f3(xs[i + 2]), f3(xs[i + 3]), nullptr);
        e += dihedral_energy(S, i, phi);
    }
    return e;
}

// Pair inclusion: |i-j| >= 3 and r^2 < rc^2 with r^2 formed in FP32 as
// fma(dz, dz, fma(dy, dy, dx dx)) (explicit round-to-nearest intrinsics, so
// the compiler cannot reassociate it; the CPU reference forms it the same way).
__device__ __forceinline__ float pair_r2(float3 d) {
    return __fmaf_rn(d.z, d.z, __fmaf_rn(d.y, d.y, __fmul_rn(d.x, d.x)));
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Lennard-Jones force on bead i from every other bead (both orders of each
// pair are evaluated, one per owning thread).
template <bool ENERGY>
__device__ __forceinline__ float3 lj_force_on(const SysDev& S, const float4* xs, int i, double& e) {
    const float3 xi = f3(xs[i]);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    float el = 0.f;
    const int N = S.N;
#pragma unroll 4
    for (int j = 0; j < N; ++j) {
        const float4 xj = xs[j];
        const float3 d = make_float3(xj.x - xi.x, xj.y - xi.y, xj.z - xi.z);
        const float r2 = pair_r2(d);
        const bool inc = (r2 < S.rc2) && (j - i > 2 || i - j > 2);
        const float inv = __fdividef(1.0f, r2);
        const float sr2 = S.sig2 * inv;
        const float sr6 = sr2 * sr2 * sr2;
        float c = S.lj_eps24 * inv * sr6 * (2.0f * sr6 - 1.0f);
        c = inc ? c : 0.0f;
        fx = fmaf(-c, d.x, fx);
        fy = fmaf(-c, d.y, fy);
        fz = fmaf(-c, d.z, fz);
        if (ENERGY) el += inc ? (S.lj_eps4 * sr6 * (sr6 - 1.0f) - S.urc) : 0.0f;
    }
    if (ENERGY) e += 0.5 * (double)el;
    return make_float3(fx, fy, fz);
}

template <typename T>
__device__ __forceinline__ T block_sum_ordered(T v, T* red) {
    // fixed-shape tree: warp shuffles, then warp 0 over the warp partials
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T r = 0;
    if (warp == 0) {
        r = lane < nw ? red[lane] : (T)0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;   // valid in warp 0
}

// ---------------------------------------------------------------------------
// Bonded terms evaluated once per term index t (bond t, angle t, dihedral t)
// into shared per-term force slots, then gathered per bead in a fixed order.
__device__ __forceinline__ void bonded_terms_to_smem(const SysDev& S, const float4* xs, int t, float3* fB, float3* fA,
                                                     float3* fD) {
    const int N = S.N;
    if (t + 1 < N) fB[t] = bond_force(S, f3(xs[t]), f3(xs[t + 1]));
    if (t + 2 < N) {
        float3 fa, fc, fb;
        angle_forces(S, f3(xs[t]), f3(xs[t + 1]), f3(xs[t + 2]), fa, fc, fb);
        fA[3 * t] = fa;
        fA[3 * t + 1] = fc;
        fA[3 * t + 2] = fb;
    }
    if (t + 3 < N) {
        float3 g[4];
        const float phi = rid_torsion(f3(xs[t]), f3(xs[t + 1]), f3(xs[t + 2]), f3(xs[t + 3]), g);
        const float m = dihedral_mdU(S, t, phi);
#pragma unroll
        for (int a = 0; a < 4; ++a) fD[4 * t + a] = m * g[a];
    }
}

__device__ __forceinline__ float3 bonded_gather(const SysDev& S, int i, const float3* fB, const float3* fA,
                                                const float3* fD) {
    const int N = S.N;
    float3 f = make_float3(0.f, 0.f, 0.f);
    if (i + 1 < N) f = f + fB[i];
    if (i >= 1) f = f - fB[i - 1];
    if (i + 2 < N) f = f + fA[3 * i];
    if (i >= 1 && i + 1 < N) f = f + fA[3 * (i - 1) + 1];
    if (i >= 2) f = f + fA[3 * (i - 2) + 2];
    if (i + 3 < N) f = f + fD[4 * i];
    if (i >= 1 && i + 2 < N) f = f + fD[4 * (i - 1) + 1];
    if (i >= 2 && i + 1 < N) f = f + fD[4 * (i - 2) + 2];
    if (i >= 3) f = f + fD[4 * (i - 3) + 3];
    return f;
}

// One Lennard-Jones interaction seen from bead i (d = x_j - x_i).  Adds
// c d with c = (1/r^2) (s/r)^6 (2 (s/r)^6 - 1) for an included pair; the
// -24 eps factor is applied once per bead.  SIG1: sigma = 1.
template <bool EXCL, bool SIG1, bool ENERGY>
__device__ __forceinline__ void lj_pair(const SysDev& S, float3 xi, float4 xj, int i, int j, float& fx, float& fy,
                                        float& fz, float& el) {
    const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
    const float r2 = pair_r2(make_float3(dx, dy, dz));
    bool inc = r2 < S.rc2;
    if (EXCL) inc = inc && (j - i > 2 || i - j > 2);
    const float inv = rcp_approx(r2);
    const float sr2 = SIG1 ? inv : S.sig2 * inv;
    const float sr6 = sr2 * sr2 * sr2;
    float c = inv * (sr6 * fmaf(2.0f, sr6, -1.0f));
    c = inc ? c : 0.0f;
    fx = fmaf(c, dx, fx);
    fy = fmaf(c, dy, fy);
    fz = fmaf(c, dz, fz);
    if (ENERGY) el += inc ? (S.lj_eps4 * sr6 * (sr6 - 1.0f) - S.urc) : 0.0f;
}

// Pair culling by bounding boxes.  Beads are grouped in clusters of 8
// consecutive beads; a warp (32 consecutive i beads) visits only the clusters
// whose box gap to the warp's own box is inside the cutoff.  The gap is formed
// with the same FP32 subtractions and the same fused r^2 as the pair test, and
// rounding is monotonic, so every pair of a skipped cluster has r^2 >= gap^2
// >= rc^2: it is one the pair test would exclude, and skipping it changes no
// result (an excluded pair adds exactly +0).
constexpr int LJ_CLUSTER = 8;
constexpr int LJ_MAX_MASK_WORDS = (RID_MAX_BEADS / LJ_CLUSTER + 31) / 32;

template <bool EXCL, bool SIG1, bool ENERGY>
__device__ __forceinline__ void lj_cluster(const SysDev& S, const float4* xj, float3 xi, int i, int j0, float& fx,
                                           float& fy, float& fz, float& el) {
#pragma unroll
    for (int k = 0; k < LJ_CLUSTER; ++k) lj_pair<EXCL, SIG1, ENERGY>(S, xi, xj[k], i, j0 + k, fx, fy, fz, el);
}

// Walk the kept clusters of one warp in increasing order; clusters that meet
// the band [b0, b1] around the warp's beads test the |i - j| > 2 exclusion.
template <bool SIG1, bool ENERGY>
__device__ __forceinline__ void lj_row_culled(const SysDev& S, const float4* xs, const unsigned* keep, int nwords,
                                              float3 xi, int i, int cb0, int cb1, float& fx, float& fy, float& fz,
                                              float& el) {
    for (int q = 0; q < nwords; ++q) {
        unsigned m = keep[q];
        while (m) {
            const int c = 32 * q + __ffs(m) - 1;
            m &= m - 1;
            const int j0 = LJ_CLUSTER * c;
            if (c >= cb0 && c <= cb1) lj_cluster<true, SIG1, ENERGY>(S, xs + j0, xi, i, j0, fx, fy, fz, el);
            else lj_cluster<false, SIG1, ENERGY>(S, xs + j0, xi, i, j0, fx, fy, fz, el);
        }
    }
}

// At most 224 threads (7 warps) and 40 registers per thread, so that seven
// CTAs (one walker each) fit on an SM.
constexpr int FF_THREADS = 224;

// Force-field forces (bonded + all-pairs LJ, culled by cluster boxes) of
// every bead at the current positions -> fff.  One CTA per walker.  BSMEM:
// bonded terms through shared per-term slots (chains up to
// RID_BONDED_SMEM_MAX beads), else per bead.
template <bool ENERGY, bool BSMEM>
__global__ void __maxnreg__(32) k_ff(SysDev S, StateDev st) {
    extern __shared__ float4 sm4[];
    __shared__ double red[32];
    __shared__ unsigned keep_s[FF_THREADS / 32][LJ_MAX_MASK_WORDS];
    const int w = blockIdx.x, N = S.N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nclus = (N + LJ_CLUSTER - 1) / LJ_CLUSTER, N8 = nclus * LJ_CLUSTER;
    const int nwords = (nclus + 31) / 32;
    float4* xs = sm4;                                         // [N8] float4, far-away padding beyond N
    float4* cbox = xs + N8;                                   // [nclus] x (lo, hi)
    float3* fB = reinterpret_cast<float3*>(cbox + 2 * nclus); // [N]  float3 (BSMEM only)
    float3* fA = fB + N;                                      // [3N]
    float3* fD = fA + 3 * N;                                  // [4N]  -> see rid_ff_smem_bytes
    const long long base = (long long)w * N;
    for (int i = threadIdx.x; i < N8; i += blockDim.x)
        xs[i] = i < N ? st.x[base + i] : make_float4(1.0e30f, 1.0e30f, 1.0e30f, 0.0f);
    __syncthreads();
    for (int c = threadIdx.x; c < nclus; c += blockDim.x) {
        const int j1 = min(LJ_CLUSTER * (c + 1), N);
        float4 lo = xs[LJ_CLUSTER * c], hi = lo;
        for (int j = LJ_CLUSTER * c + 1; j < j1; ++j) {
            const float4 p = xs[j];
            lo.x = fminf(lo.x, p.x); lo.y = fminf(lo.y, p.y); lo.z = fminf(lo.z, p.z);
            hi.x = fmaxf(hi.x, p.x); hi.y = fmaxf(hi.y, p.y); hi.z = fmaxf(hi.z, p.z);
        }
        cbox[2 * c] = lo;
        cbox[2 * c + 1] = hi;
    }
    if (BSMEM) {
        for (int t = threadIdx.x; t < N; t += blockDim.x) bonded_terms_to_smem(S, xs, t, fB, fA, fD);
    }
    __syncthreads();
    const bool sig1 = S.sig2 == 1.0f;
    double e = 0.0;
    const int iters = (N + blockDim.x - 1) / blockDim.x;
    for (int it = 0; it < iters; ++it) {
        const int i = it * blockDim.x + threadIdx.x;
        const int wlo = i - lane, whi = wlo + 31;
        if (wlo >= N) break;                                  // warp-uniform: no bead of this warp
        const bool act = i < N;
        const float3 xi = f3(xs[act ? i : N - 1]);
        // the warp's box (lanes past N repeat bead N - 1, which is in the warp)
        float3 ilo = xi, ihi = xi;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ilo.x = fminf(ilo.x, __shfl_xor_sync(0xffffffffu, ilo.x, o));
            ilo.y = fminf(ilo.y, __shfl_xor_sync(0xffffffffu, ilo.y, o));
            ilo.z = fminf(ilo.z, __shfl_xor_sync(0xffffffffu, ilo.z, o));
            ihi.x = fmaxf(ihi.x, __shfl_xor_sync(0xffffffffu, ihi.x, o));
            ihi.y = fmaxf(ihi.y, __shfl_xor_sync(0xffffffffu, ihi.y, o));
            ihi.z = fmaxf(ihi.z, __shfl_xor_sync(0xffffffffu, ihi.z, o));
        }
        for (int q = 0; q < nwords; ++q) {
            const int c = 32 * q + lane;
            bool kp = false;
            if (c < nclus) {
                const float4 lo = cbox[2 * c], hi = cbox[2 * c + 1];
                const float gx = fmaxf(0.0f, fmaxf(lo.x - ihi.x, ilo.x - hi.x));
                const float gy = fmaxf(0.0f, fmaxf(lo.y - ihi.y, ilo.y - hi.y));
                const float gz = fmaxf(0.0f, fmaxf(lo.z - ihi.z, ilo.z - hi.z));
                kp = !(pair_r2(make_float3(gx, gy, gz)) >= S.rc2);
            }
            const unsigned b = __ballot_sync(0xffffffffu, kp);
            if (lane == 0) keep_s[warp][q] = b;
        }
        __syncwarp();
        const int b0 = wlo - 2 > 0 ? wlo - 2 : 0;
        const int b1 = whi + 2 < N - 1 ? whi + 2 : N - 1;
        float fx = 0.f, fy = 0.f, fz = 0.f, el = 0.f;
        if (sig1)
            lj_row_culled<true, ENERGY>(S, xs, keep_s[warp], nwords, xi, i, b0 / LJ_CLUSTER, b1 / LJ_CLUSTER, fx, fy,
                                        fz, el);
        else
            lj_row_culled<false, ENERGY>(S, xs, keep_s[warp], nwords, xi, i, b0 / LJ_CLUSTER, b1 / LJ_CLUSTER, fx,
                                         fy, fz, el);
        __syncwarp();                                         // keep_s is rewritten by the next iteration
        if (act) {
            const float3 fb = BSMEM ? bonded_gather(S, i, fB, fA, fD) : bonded_force_on(S, xs, i);
            const float s = -S.lj_eps24;
            st.fff[base + i] = make_float4(fmaf(s, fx, fb.x), fmaf(s, fy, fb.y), fmaf(s, fz, fb.z), 0.0f);
            if (ENERGY) e += 0.5 * (double)el + bonded_energy_from(S, xs, i);
        }
    }
    if (ENERGY) {
        const double tot = block_sum_ordered<double>(e, red);
        if (threadIdx.x == 0) st.eff[w] = tot;
    }
}

// ---------------------------------------------------------------------------
// k_head: the closing half of step t-1 (CV force from the ensemble or the
// restraint, chain rule through the torsion Jacobians, B half-kick, traces and
// FP64 label sums) fused with the opening half of step t (B A O A) and the
// CVs at the new positions.
//   FIN: finish the previous evaluation (f = fff + sum_j F_s,j ds_j/dx)
//   KICK: apply the closing half-kick of the previous step (FIN only)
//   INT: 0 nothing, 1 CVs at the current positions, 2 B-A-O-A then CVs
// With FIN and INT = 0 the total force is stored (end of a call); with
// FIN = 0 the opening kick uses the stored force.
constexpr int HEAD_THREADS = 128;  // four warps per walker, seven CTAs per SM: the grid is resident at once
constexpr int HEAD_BEADS = 2;      // beads per thread per batch, loaded before they are needed

template <int MODE, bool FIN, bool KICK, int INT, bool ENERGY>
__global__ void __launch_bounds__(HEAD_THREADS, 7) k_head(SysDev S, StateDev st, EnsDev E, LabelDev lab, long long t_fin,
                                                        int slot, float* __restrict__ cv_out,
                                                        float* __restrict__ eps_out, double* __restrict__ energy_out,
                                                        long long T, uint32_t step) {
    extern __shared__ float4 xs[];
    __shared__ float Fs[RID_MAX_CV];
    __shared__ float s_eps, s_abar;
    __shared__ double red[32];
    const int w = blockIdx.x, N = S.N, C = S.C, W = st.W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long base = (long long)w * N;
    const float kick = S.half_dt * S.inv_mass;
    constexpr int BATCH = HEAD_THREADS * HEAD_BEADS;
    // bead data of the first batch (and its Langevin noise) is loaded / drawn
    // before the ensemble reduction, so the two overlap
    float3 px[HEAD_BEADS], pv[HEAD_BEADS], pf[HEAD_BEADS], pz[HEAD_BEADS];
    auto load_batch = [&](int b0) {
#pragma unroll
        for (int k = 0; k < HEAD_BEADS; ++k) {
            const int i = b0 + k * HEAD_THREADS + threadIdx.x;
            if (i < N) {
                px[k] = f3(st.x[base + i]);
                pv[k] = f3(st.v[base + i]);
                if (FIN) pf[k] = f3(st.fff[base + i]);
                else if (INT == 2) pf[k] = f3(st.f[base + i]);
                if (INT == 2 && S.c2 != 0.0f) pz[k] = rid_normals3(rid_philox(make_uint4(i, w, step, 0u), S.key0, S.key1));
            }
        }
    };
    load_batch(0);
    if (FIN) {
        if (MODE == 1) {
            if (warp == 0) {
                const float invM = 1.0f / (float)E.M;
                // member values: lane k holds entries k and k + 32 of [M][aslices]
                const int na = E.M * E.aslices;
                float av = 0.0f;
                for (int k = lane; k < na; k += 32) av += st.Aval[(long long)k * W + w];
                float d2 = 0.0f;
                for (int j = lane; j < C; j += 32) {
                    float fb = 0.0f;
                    for (int m = 0; m < E.M; ++m) fb += st.gradA[((long long)m * W + w) * C + j];
                    fb *= invM;
                    for (int m = 0; m < E.M; ++m) {
                        const float d = st.gradA[((long long)m * W + w) * C + j] - fb;
                        d2 = fmaf(d, d, d2);
                    }
                    Fs[j] = fb;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
                    av += __shfl_xor_sync(0xffffffffu, av, o);
                }
                const float eps = sqrtf(d2 * invM);
                float sig;
                if (eps < E.e0) sig = 1.0f;
                else if (eps >= E.e1) sig = 0.0f;
                else sig = 0.5f * (1.0f + cospif((eps - E.e0) / (E.e1 - E.e0)));
                __syncwarp();
                for (int j = lane; j < C; j += 32) Fs[j] *= sig;
                if (lane == 0) {
                    s_abar = av * invM;
                    s_eps = eps;
                    st.eps[w] = eps;
                }
            }
        } else if (MODE == 2) {
            const bool sample = KICK && t_fin >= lab.n_equil;
            long long b = 0;
            if (sample) b = ((t_fin - lab.n_equil) * lab.B) / lab.K;
            for (int j = threadIdx.x; j < C; j += blockDim.x) {
                const long long o = (long long)w * C + j;
                const double d = rid_wrapd((double)st.s[o] - lab.s0[o]);
                Fs[j] = (float)(-lab.kappa[o] * d);
                if (sample) {
                    lab.sum[o] += d;
                    lab.sum2[o] = fma(d, d, lab.sum2[o]);
                    lab.bsum[o * lab.B + b] += d;
                }
            }
            if (threadIdx.x == 0) { s_eps = 0.0f; s_abar = 0.0f; }
        } else {
            for (int j = threadIdx.x; j < C; j += blockDim.x) Fs[j] = 0.0f;
            if (threadIdx.x == 0) { s_eps = 0.0f; s_abar = 0.0f; }
        }
        __syncthreads();
        // traces of the finished step read the CVs before they are recomputed
        if (slot >= 0) {
            if (cv_out)
                for (int j = threadIdx.x; j < C; j += blockDim.x)
                    cv_out[((long long)w * T + slot) * C + j] = st.s[(long long)w * C + j];
            if (eps_out && threadIdx.x == 0) eps_out[(long long)w * T + slot] = s_eps;
        }
    }
    double ke = 0.0;
    int bad = 0;
    for (int b0 = 0; b0 < N; b0 += BATCH) {
        if (b0 > 0) load_batch(b0);
#pragma unroll
        for (int k = 0; k < HEAD_BEADS; ++k) {
            const int i = b0 + k * HEAD_THREADS + threadIdx.x;
            if (i >= N) break;
            float4 x = make_float4(px[k].x, px[k].y, px[k].z, 0.f);
            float4 v = make_float4(pv[k].x, pv[k].y, pv[k].z, 0.f);
            float4 f = make_float4(pf[k].x, pf[k].y, pf[k].z, 0.f);
            if (FIN) {
                for (int e = S.acv_off[i]; e < S.acv_off[i + 1]; ++e) {
                    const int2 ja = S.acv[e];
                    const float4 g = st.J[((long long)w * C + ja.x) * 4 + ja.y];
                    const float fs = Fs[ja.x];
                    f.x = fmaf(fs, g.x, f.x);
                    f.y = fmaf(fs, g.y, f.y);
                    f.z = fmaf(fs, g.z, f.z);
                }
                bad |= !(isfinite(f.x) && isfinite(f.y) && isfinite(f.z));
                if (KICK) {
                    v.x = fmaf(kick, f.x, v.x);
                    v.y = fmaf(kick, f.y, v.y);
                    v.z = fmaf(kick, f.z, v.z);
                    bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z));
                    if (ENERGY)
                        ke += 0.5 / (double)S.inv_mass * ((double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z);
                }
                if (INT != 2) st.f[base + i] = f;
            }
            if (INT == 2) {
                v.x = fmaf(kick, f.x, v.x);             // B
                v.y = fmaf(kick, f.y, v.y);
                v.z = fmaf(kick, f.z, v.z);
                x.x = fmaf(S.half_dt, v.x, x.x);        // A
                x.y = fmaf(S.half_dt, v.y, x.y);
                x.z = fmaf(S.half_dt, v.z, x.z);
                if (S.c2 != 0.0f) {                     // O
                    const float3 z = pz[k];
                    v.x = fmaf(S.c1, v.x, S.c2 * z.x);
                    v.y = fmaf(S.c1, v.y, S.c2 * z.y);
                    v.z = fmaf(S.c1, v.z, S.c2 * z.z);
                }
                x.x = fmaf(S.half_dt, v.x, x.x);        // A
                x.y = fmaf(S.half_dt, v.y, x.y);
                x.z = fmaf(S.half_dt, v.z, x.z);
                st.x[base + i] = x;
            }
            if (INT == 2 || (FIN && KICK)) st.v[base + i] = v;
            if (INT != 0) xs[i] = x;
        }
    }
    if (FIN) {
        if (bad) st.flags[w] = 1;
        if (ENERGY) {
            const double kt = block_sum_ordered<double>(ke, red);
            if (threadIdx.x == 0 && slot >= 0 && energy_out) {
                double* e = energy_out + ((long long)w * T + slot) * 3;
                e[0] = st.eff[w];
                e[1] = (MODE == 1) ? -(double)s_abar : 0.0;
                e[2] = kt;
            }
        }
    }
    if (INT != 0) {
        __syncthreads();   // all Jacobian reads of the finish are done; positions staged
        for (int j = threadIdx.x; j < C; j += blockDim.x) {
            const int4 q = S.cv[j];
            float3 g[4];
            const float sj = rid_torsion(f3(xs[q.x]), f3(xs[q.y]), f3(xs[q.z]), f3(xs[q.w]), g);
            const long long o = (long long)w * C + j;
            st.s[o] = sj;
#pragma unroll
            for (int a = 0; a < 4; ++a) st.J[o * 4 + a] = make_float4(g[a].x, g[a].y, g[a].z, 0.0f);
            float sn, cs;
            sincosf(sj, &sn, &cs);
            st.u[(long long)w * 2 * C + 2 * j] = cs;
            st.u[(long long)w * 2 * C + 2 * j + 1] = sn;
        }
    }
}

// Pair-inclusion bit mask of the force kernel's LJ loop.
__global__ void __launch_bounds__(256) k_pair_mask(SysDev S, StateDev st, uint32_t* __restrict__ mask) {
    extern __shared__ float4 xs[];
    const int w = blockIdx.x, N = S.N, nw = (N + 31) >> 5;
    for (int i = threadIdx.x; i < N; i += blockDim.x) xs[i] = st.x[(long long)w * N + i];
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const float3 xi = f3(xs[i]);
        for (int jw = 0; jw < nw; ++jw) {
            uint32_t bits = 0;
            for (int b = 0; b < 32; ++b) {
                const int j = jw * 32 + b;
                if (j >= N) break;
                const float4 xj = xs[j];
                const float r2 = pair_r2(make_float3(xj.x - xi.x, xj.y - xi.y, xj.z - xi.z));
                if ((r2 < S.rc2) && (j - i > 2 || i - j > 2)) bits |= 1u << b;
            }
            mask[((long long)w * N + i) * nw + jw] = bits;
        }
    }
}

__global__ void k_label_final(LabelDev lab, int W, int C, double* __restrict__ mf, double* __restrict__ se,
                              double* __restrict__ sd) {
    const long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= (long long)W * C) return;
    const double K = (double)lab.K, kap = lab.kappa[o];
    const double mean = lab.sum[o] / K;
    double var = lab.sum2[o] / K - mean * mean;
    if (var < 0) var = 0;
    const int B = lab.B;
    double bm_mean = 0.0;
    for (int b = 0; b < B; ++b) {
        const long long lo = (b * lab.K + B - 1) / B, hi = ((b + 1) * lab.K + B - 1) / B;
        bm_mean += lab.bsum[o * B + b] / (double)(hi - lo) / B;
    }
    double ss = 0.0;
    for (int b = 0; b < B; ++b) {
        const long long lo = (b * lab.K + B - 1) / B, hi = ((b + 1) * lab.K + B - 1) / B;
        const double d = lab.bsum[o * B + b] / (double)(hi - lo) - bm_mean;
        ss += d * d;
    }
    mf[o] = -kap * mean;
    se[o] = kap * sqrt(ss / (B - 1) / B);
    sd[o] = kap * sqrt(var);
}

__global__ void k_philox(long long n, const uint32_t* __restrict__ ctr, uint32_t k0, uint32_t k1,
                         uint32_t* __restrict__ words, float* __restrict__ normals) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint4 o = rid_philox(c, k0, k1);
    if (words) {
        words[4 * i] = o.x;
        words[4 * i + 1] = o.y;
        words[4 * i + 2] = o.z;
        words[4 * i + 3] = o.w;
    }
    if (normals) {
        const float3 z = rid_normals3(o);
        normals[3 * i] = z.x;
        normals[3 * i + 1] = z.y;
        normals[3 * i + 2] = z.z;
    }
}

inline int chain_threads(int N) {
    int t = ((N + 31) / 32) * 32;
    return t > 256 ? 256 : (t < 32 ? 32 : t);
}

}  // namespace

// ---------------------------------------------------------------------------
void rid_launch_pack(const float* src, float4* dst, long long n, cudaStream_t s) {
    if (n > 0) k_pack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
}
void rid_launch_unpack(const float4* src, float* dst, long long n, cudaStream_t s) {
    if (n > 0) k_unpack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
}
void rid_launch_mb(const SysDev& S, StateDev st, int W, uint32_t step0, cudaStream_t s) {
    const long long n = (long long)W * S.N;
    if (n > 0) k_mb<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(S, st, W, step0);
}
void rid_launch_pair_mask(const SysDev& S, StateDev st, int W, uint32_t* mask, cudaStream_t s) {
    static bool attr = false;   // positions of up to RID_MAX_BEADS beads exceed the default 48 KB
    if (!attr) {
        cudaFuncSetAttribute(k_pair_mask, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    k_pair_mask<<<W, chain_threads(S.N), sizeof(float4) * (size_t)S.N, s>>>(S, st, mask);
}

// Shared memory of k_ff: positions [N8] float4 (N8 = N rounded up to the
// 8-bead cluster), cluster boxes [N8 / 8][2] float4 and, with per-term bonded
// slots, bond [N] + angle [3N] + dihedral [4N] forces as float3.
int rid_ff_smem_bytes(int N) {
    const size_t nclus = (size_t)(N + LJ_CLUSTER - 1) / LJ_CLUSTER;
    return (int)(sizeof(float4) * (nclus * LJ_CLUSTER + 2 * nclus) +
                 (N <= RID_BONDED_SMEM_MAX ? sizeof(float3) * 8 * (size_t)N : 0));
}

void rid_launch_ff(const SysDev& S, StateDev st, int W, bool energy, cudaStream_t s) {
    const int th = chain_threads(S.N) < FF_THREADS ? chain_threads(S.N) : FF_THREADS;
    const size_t sm = (size_t)rid_ff_smem_bytes(S.N);
    const bool bsm = S.N <= RID_BONDED_SMEM_MAX;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_ff<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_ff<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_ff<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_ff<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    if (bsm) {
        if (energy) k_ff<true, true><<<W, th, sm, s>>>(S, st);
        else k_ff<false, true><<<W, th, sm, s>>>(S, st);
    } else {
        if (energy) k_ff<true, false><<<W, th, sm, s>>>(S, st);
        else k_ff<false, false><<<W, th, sm, s>>>(S, st);
    }
}

template <int MODE, bool FIN, bool KICK, int INT>
static void head_e(const HeadArgs& a, cudaStream_t s) {
    const int th = HEAD_THREADS;
    const size_t sm = sizeof(float4) * (size_t)a.S.N;
    static bool attr = false;   // positions of up to RID_MAX_BEADS beads exceed the default 48 KB
    if (!attr) {
        cudaFuncSetAttribute(k_head<MODE, FIN, KICK, INT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             sizeof(float4) * RID_MAX_BEADS);
        cudaFuncSetAttribute(k_head<MODE, FIN, KICK, INT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             sizeof(float4) * RID_MAX_BEADS);
        attr = true;
    }
    if (a.energy)
        k_head<MODE, FIN, KICK, INT, true><<<a.W, th, sm, s>>>(a.S, a.st, a.E, a.lab, a.t_fin, a.slot, a.cv_out,
                                                                 a.eps_out, a.energy_out, a.T, a.step);
    else
        k_head<MODE, FIN, KICK, INT, false><<<a.W, th, sm, s>>>(a.S, a.st, a.E, a.lab, a.t_fin, a.slot, a.cv_out,
                                                                  a.eps_out, a.energy_out, a.T, a.step);
}

template <int MODE>
static void head_m(const HeadArgs& a, cudaStream_t s) {
    // (FIN, KICK, INT) combinations used by the driver
    if (!a.fin && a.integ == 1) head_e<MODE, false, false, 1>(a, s);
    else if (!a.fin && a.integ == 2) head_e<MODE, false, false, 2>(a, s);
    else if (a.fin && a.kick && a.integ == 2) head_e<MODE, true, true, 2>(a, s);
    else if (a.fin && a.kick && a.integ == 0) head_e<MODE, true, true, 0>(a, s);
    else if (a.fin && !a.kick && a.integ == 0) head_e<MODE, true, false, 0>(a, s);
    else head_e<MODE, true, false, 2>(a, s);
}

void rid_launch_head(const HeadArgs& a, cudaStream_t s) {
    if (a.mode == 1) head_m<1>(a, s);
    else if (a.mode == 2) head_m<2>(a, s);
    else head_m<0>(a, s);
}

void rid_launch_label_final(const LabelDev& lab, int W, int C, double* mf, double* se, double* sd, cudaStream_t s) {
    const long long n = (long long)W * C;
    if (n > 0) k_label_final<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(lab, W, C, mf, se, sd);
}

void rid_launch_philox(long long n, const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* words, float* normals,
                       cudaStream_t s) {
    if (n > 0) k_philox<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, ctr, k0, k1, words, normals);
}
