// rid_forces.cuh -- force-field device functions shared by the per-step
// kernels (k_step.cu) and the persistent label kernel (k_label_fused.cu).
// Bonded terms (harmonic bonds and angles, 3-term cosine dihedrals), the
// Lennard-Jones pair interaction with cluster-box culling, and an ordered
// block reduction.  Every sum is taken in a fixed order.
#pragma once

#include "rid_internal.cuh"

namespace {

// ---------------------------------------------------------------------------
// Bonded terms, gathered per bead (each term is evaluated by every bead it
// touches, which keeps the sums ordered and needs no atomics).

// Force on p from the harmonic bond p-q.
__device__ __forceinline__ float3 bond_force(const SysDev& S, float3 p, float3 q) {
    const float3 d = q - p;
    const float r = sqrtf(dot3(d, d));
    return (S.kb * (r - S.r0) / r) * d;
}

// Harmonic angle a-c-b (vertex c): forces on a, c, b.  Written with
// explicitly rounded operations so that the compiler fuses nothing: callers
// that use only one of the three forces get the same bits as callers that use
// all of them.
__device__ __forceinline__ void angle_forces(const SysDev& S, float3 pa, float3 pc, float3 pb, float3& fa,
                                             float3& fc, float3& fb) {
    const float3 a = pa - pc, b = pb - pc;
    const float3 axb = make_float3(__fsub_rn(__fmul_rn(a.y, b.z), __fmul_rn(a.z, b.y)),
                                   __fsub_rn(__fmul_rn(a.z, b.x), __fmul_rn(a.x, b.z)),
                                   __fsub_rn(__fmul_rn(a.x, b.y), __fmul_rn(a.y, b.x)));
    const float cr = sqrtf(dot3(axb, axb)), dp = dot3(a, b);
    const float th = atan2f(cr, dp);
    const float dU = __fmul_rn(S.ka, __fsub_rn(th, S.th0));
    const float ia = __fdiv_rn(1.0f, cr);
    const float qa = __fdiv_rn(dp, dot3(a, a)), qb = __fdiv_rn(dp, dot3(b, b));
    // d theta / d a and d theta / d b
    const float3 ga = make_float3(__fmul_rn(ia, __fsub_rn(__fmul_rn(qa, a.x), b.x)),
                                  __fmul_rn(ia, __fsub_rn(__fmul_rn(qa, a.y), b.y)),
                                  __fmul_rn(ia, __fsub_rn(__fmul_rn(qa, a.z), b.z)));
    const float3 gb = make_float3(__fmul_rn(ia, __fsub_rn(__fmul_rn(qb, b.x), a.x)),
                                  __fmul_rn(ia, __fsub_rn(__fmul_rn(qb, b.y), a.y)),
                                  __fmul_rn(ia, __fsub_rn(__fmul_rn(qb, b.z), a.z)));
    const float m = -dU;
    fa = make_float3(__fmul_rn(m, ga.x), __fmul_rn(m, ga.y), __fmul_rn(m, ga.z));
    fb = make_float3(__fmul_rn(m, gb.x), __fmul_rn(m, gb.y), __fmul_rn(m, gb.z));
    fc = make_float3(__fmul_rn(dU, __fadd_rn(ga.x, gb.x)), __fmul_rn(dU, __fadd_rn(ga.y, gb.y)),
                     __fmul_rn(dU, __fadd_rn(ga.z, gb.z)));
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
// LANE: before a cluster's pairs, each lane tests its own bead against the
// cluster box (the same gap and fused r^2 as the warp mask); a cluster that no
// lane's bead can reach is skipped whole -- exact for the same reason as the
// mask, so kernels with and without the test give the same bits.  It pays in
// the chain-resident label kernels (batching +6%), not in k_ff.
template <bool SIG1, bool ENERGY, bool LANE = false>
__device__ __forceinline__ void lj_row_culled(const SysDev& S, const float4* xs, const float4* cbox,
                                              const unsigned* keep, int nwords, float3 xi, int i, int cb0, int cb1,
                                              float& fx, float& fy, float& fz, float& el) {
    for (int q = 0; q < nwords; ++q) {
        unsigned m = keep[q];
        while (m) {
            const int c = 32 * q + __ffs(m) - 1;
            m &= m - 1;
            if (LANE) {
                const float4 lo = cbox[2 * c], hi = cbox[2 * c + 1];
                const float gx = fmaxf(0.0f, fmaxf(lo.x - xi.x, xi.x - hi.x));
                const float gy = fmaxf(0.0f, fmaxf(lo.y - xi.y, xi.y - hi.y));
                const float gz = fmaxf(0.0f, fmaxf(lo.z - xi.z, xi.z - hi.z));
                if (!__any_sync(0xffffffffu, !(pair_r2(make_float3(gx, gy, gz)) >= S.rc2))) continue;
            }
            const int j0 = LJ_CLUSTER * c;
            if (c >= cb0 && c <= cb1) lj_cluster<true, SIG1, ENERGY>(S, xs + j0, xi, i, j0, fx, fy, fz, el);
            else lj_cluster<false, SIG1, ENERGY>(S, xs + j0, xi, i, j0, fx, fy, fz, el);
        }
    }
}

// Bonded force on bead i in the order of bonded_gather: bonds and angles are
// recomputed here, the dihedral terms come from the shared slots fD written by
// bonded_dihedrals_to_smem.  Adds are non-contractible, so the result is
// bit-identical to the all-slot path.
__device__ __forceinline__ float3 add3_rn(float3 a, float3 b) {
    return make_float3(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z));
}
__device__ __forceinline__ float3 sub3_rn(float3 a, float3 b) {
    return make_float3(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z));
}

__device__ __forceinline__ void bonded_dihedrals_to_smem(const SysDev& S, const float4* xs, int t, float3* fD) {
    if (t + 3 < S.N) {
        float3 g[4];
        const float phi = rid_torsion(f3(xs[t]), f3(xs[t + 1]), f3(xs[t + 2]), f3(xs[t + 3]), g);
        const float m = dihedral_mdU(S, t, phi);
#pragma unroll
        for (int a = 0; a < 4; ++a) fD[4 * t + a] = m * g[a];
    }
}

__device__ float3 bonded_gather_hybrid(const SysDev& S, const float4* xs, int i, const float3* fD) {
    const int N = S.N;
    float3 f = make_float3(0.f, 0.f, 0.f);
    float3 fa, fc, fb;
    if (i + 1 < N) f = add3_rn(f, bond_force(S, f3(xs[i]), f3(xs[i + 1])));
    if (i >= 1) f = sub3_rn(f, bond_force(S, f3(xs[i - 1]), f3(xs[i])));
    if (i + 2 < N) {
        angle_forces(S, f3(xs[i]), f3(xs[i + 1]), f3(xs[i + 2]), fa, fc, fb);
        f = add3_rn(f, fa);
    }
    if (i >= 1 && i + 1 < N) {
        angle_forces(S, f3(xs[i - 1]), f3(xs[i]), f3(xs[i + 1]), fa, fc, fb);
        f = add3_rn(f, fc);
    }
    if (i >= 2) {
        angle_forces(S, f3(xs[i - 2]), f3(xs[i - 1]), f3(xs[i]), fa, fc, fb);
        f = add3_rn(f, fb);
    }
    if (i + 3 < N) f = add3_rn(f, fD[4 * i]);
    if (i >= 1 && i + 2 < N) f = add3_rn(f, fD[4 * (i - 1) + 1]);
    if (i >= 2 && i + 1 < N) f = add3_rn(f, fD[4 * (i - 2) + 2]);
    if (i >= 3) f = add3_rn(f, fD[4 * (i - 3) + 3]);
    return f;
}

// Restrained-MD statistics of one (run, CV) entry o from the FP64 sums:
// MF = -kappa mean(d), SE = kappa std_ddof1(block means) / sqrt(B) with sample
// k of K in block floor(k B / K), std = kappa population std of d.
__device__ __forceinline__ void label_stats(const double* sum, const double* sum2, const double* bsum, double kap,
                                            long long Kl, int B, double& mf, double& se, double& sd) {
    const double K = (double)Kl;
    const double mean = *sum / K;
    double var = *sum2 / K - mean * mean;
    if (var < 0) var = 0;
    double bm_mean = 0.0;
    for (int b = 0; b < B; ++b) {
        const long long lo = (b * Kl + B - 1) / B, hi = ((b + 1) * Kl + B - 1) / B;
        bm_mean += bsum[b] / (double)(hi - lo) / B;
    }
    double ss = 0.0;
    for (int b = 0; b < B; ++b) {
        const long long lo = (b * Kl + B - 1) / B, hi = ((b + 1) * Kl + B - 1) / B;
        const double d = bsum[b] / (double)(hi - lo) - bm_mean;
        ss += d * d;
    }
    mf = -kap * mean;
    se = kap * sqrt(ss / (B - 1) / B);
    sd = kap * sqrt(var);
}

// The warp's keep mask over 8-bead clusters: bit c of word q is set when
// cluster 32 q + c may hold a pair inside the cutoff for some bead of the
// warp (lanes past the last bead repeat bead N - 1, which is in the warp).
__device__ __forceinline__ void lj_warp_keep_masks(const SysDev& S, const float4* cbox, int nclus, float3 xi,
                                                   unsigned* keep) {
    const int lane = threadIdx.x & 31;
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
    const int nwords = (nclus + 31) / 32;
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
        const unsigned bits = __ballot_sync(0xffffffffu, kp);
        if (lane == 0) keep[q] = bits;
    }
    __syncwarp();
}

// Bounding boxes of the 8-bead clusters (positions padded to a multiple of 8).
__device__ __forceinline__ void lj_cluster_boxes(const float4* xs, int N, float4* cbox) {
    const int nclus = (N + LJ_CLUSTER - 1) / LJ_CLUSTER;
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
}

}  // namespace
