// k_step.cu -- per-walker kernels of the RiD Langevin step on sm_103a.
//
// One CTA owns one walker (bead chain) for the whole evaluation: the chain's
// positions are staged once in shared memory and every force term reads them
// from there.  All sums are taken in a fixed order, so results are
// bit-reproducible run to run.
//
//   k_ff    : force field (bonds, angles, dihedrals, cluster-culled all-pairs
//             Lennard-Jones) at the current positions
//   k_head  : CV force of the previous evaluation (ensemble bias with the
//             trust-level switch, or a harmonic restraint with FP64 label
//             sums) chain-ruled to the beads, the closing B half-kick, traces,
//             then B A O A of the next step and the torsion CVs
//   k_mb, k_pack, k_unpack, k_pair_mask, k_label_final, k_philox: helpers
#include <math.h>

#include "rid_forces.cuh"

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

// At most 224 threads (7 warps) per CTA (one walker).  k_ff gets 56 registers
// per thread (five CTAs per SM): with fewer, the unrolled pair loop cannot hold
// a cluster's positions in flight and waits on every shared-memory load
// (measured: 32 registers 35.3 us alone, 40 registers 31.5 us, 56 registers
// 30.2 us for 1024 walkers x 200 beads).
constexpr int FF_THREADS = 224;

// Force-field forces (bonded + all-pairs LJ, culled by cluster boxes) of
// every bead at the current positions -> fff.  P CTAs per walker (CTA
// w * P + p): each loads the walker's chain and cluster boxes and computes the
// forces of its ipc passes of blockDim beads (passes p * ipc ..), so a bead's
// force is the same code and order whatever P (P = 1 for energy launches,
// whose per-walker sum is over every pass).  BSMEM: bonded terms through shared
// per-term slots (chains up to RID_BONDED_SMEM_MAX beads), else per bead.
template <bool ENERGY, bool BSMEM>
__global__ void __maxnreg__(56) k_ff(SysDev S, StateDev st, int P, int ipc) {
    extern __shared__ float4 sm4[];
    __shared__ double red[32];
    __shared__ unsigned keep_s[FF_THREADS / 32][LJ_MAX_MASK_WORDS];
    const int w = blockIdx.x / P, N = S.N;
    const int p0 = (blockIdx.x - w * P) * ipc;
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
    lj_cluster_boxes(xs, N, cbox);
    if (BSMEM) {
        for (int t = threadIdx.x; t < N; t += blockDim.x) bonded_terms_to_smem(S, xs, t, fB, fA, fD);
    }
    __syncthreads();
    const bool sig1 = S.sig2 == 1.0f;
    double e = 0.0;
    const int iters = (N + blockDim.x - 1) / blockDim.x;
    const int it1 = p0 + ipc < iters ? p0 + ipc : iters;
    for (int it = p0; it < it1; ++it) {
        const int i = it * blockDim.x + threadIdx.x;
        const int wlo = i - lane, whi = wlo + 31;
        if (wlo >= N) break;                                  // warp-uniform: no bead of this warp
        const bool act = i < N;
        const float3 xi = f3(xs[act ? i : N - 1]);
        lj_warp_keep_masks(S, cbox, nclus, xi, keep_s[warp]);
        const int b0 = wlo - 2 > 0 ? wlo - 2 : 0;
        const int b1 = whi + 2 < N - 1 ? whi + 2 : N - 1;
        float fx = 0.f, fy = 0.f, fz = 0.f, el = 0.f;
        if (sig1)
            lj_row_culled<true, ENERGY>(S, xs, cbox, keep_s[warp], nwords, xi, i, b0 / LJ_CLUSTER, b1 / LJ_CLUSTER, fx, fy,
                                        fz, el);
        else
            lj_row_culled<false, ENERGY>(S, xs, cbox, keep_s[warp], nwords, xi, i, b0 / LJ_CLUSTER, b1 / LJ_CLUSTER, fx,
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
// P CTAs per walker (a thread-block cluster, P > 1 only without ENERGY): CTA p
// integrates its slice of bead batches and keeps the new positions in its
// shared memory; after a cluster barrier it forms its share of the CVs,
// reading atoms of other slices from their CTAs' shared memory.  Every CTA
// forms the CV force (the same arithmetic); CTA 0 alone writes the traces, eps
// and the label sums.  A bead's update and a CV are the same arithmetic
// whatever P.
// Thread-block cluster helpers of the split k_head: a barrier over the
// cluster's CTAs, and a float4 of a peer CTA's shared memory.
__device__ __forceinline__ void head_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ float4 head_ld_peer(const float4* local, uint32_t rank) {
    uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(local)), r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(r)
                 : "memory");
    return v;
}

constexpr int HEAD_THREADS = 128;  // four warps per walker, seven CTAs per SM: the grid is resident at once
constexpr int HEAD_BEADS = 2;      // beads per thread per batch, loaded before they are needed

template <int MODE, bool FIN, bool KICK, int INT, bool ENERGY>
__global__ void __launch_bounds__(HEAD_THREADS, 7) k_head(SysDev S, StateDev st, EnsDev E, LabelDev lab, long long t_fin,
                                                        int slot, float* __restrict__ cv_out,
                                                        float* __restrict__ eps_out, double* __restrict__ energy_out,
                                                        long long T, uint32_t step, int P) {
    extern __shared__ float4 xs[];                     // [N] positions, then (FIN) [4C] Jacobian rows, [4C] slots
    __shared__ float Fs[RID_MAX_CV];
    __shared__ float s_eps, s_abar;
    __shared__ double red[32];
    const int w = blockIdx.x / P, N = S.N, C = S.C, W = st.W;
    const int p = blockIdx.x - w * P;                      // rank in the walker's cluster
    float4* Jsm = xs + N;                                   // this walker's torsion Jacobians [C][4]
    int2* acv_s = reinterpret_cast<int2*>(Jsm + 4 * C);     // (cv, slot) list of the chain rule
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long base = (long long)w * N;
    const float kick = S.half_dt * S.inv_mass;
    const uint32_t stp = step + ((INT == 2 && st.stepbase) ? *st.stepbase : 0u);
    constexpr int BATCH = HEAD_THREADS * HEAD_BEADS;
    const int bpc = ((N + BATCH - 1) / BATCH + P - 1) / P;  // bead batches per CTA
    const int bb0 = p * bpc * BATCH, bb1 = min(N, (p + 1) * bpc * BATCH);
    // bead data of the first batch (and its Langevin noise) is loaded / drawn
    // before the ensemble reduction, so the two overlap
    float3 px[HEAD_BEADS], pv[HEAD_BEADS], pf[HEAD_BEADS], pz[HEAD_BEADS];
    int a0[HEAD_BEADS], a1[HEAD_BEADS];                    // chain-rule list range of each bead
    auto load_batch = [&](int b0) {
#pragma unroll
        for (int k = 0; k < HEAD_BEADS; ++k) {
            const int i = b0 + k * HEAD_THREADS + threadIdx.x;
            if (i < N) {
                px[k] = f3(st.x[base + i]);
                pv[k] = f3(st.v[base + i]);
                if (FIN) {
                    pf[k] = f3(st.fff[base + i]);
                    a0[k] = __ldg(S.acv_off + i);
                    a1[k] = __ldg(S.acv_off + i + 1);
                }
                else if (INT == 2) pf[k] = f3(st.f[base + i]);
                if (INT == 2 && S.c2 != 0.0f) pz[k] = rid_normals3(rid_philox(make_uint4(i, w, stp, 0u), S.key0, S.key1));
            }
        }
    };
    // warp 0 forms the CV force: it issues the member gradients of its first
    // CVs (ensembles of up to 8 members) and the member values before drawing
    // its noise, so their latency overlaps the Philox work
    constexpr int PM = 8;
    float gpre[PM];
    float avpre = 0.0f;
    const bool pre = FIN && MODE == 1 && warp == 0 && E.M <= PM;
    if (pre) {
        for (int k = lane; k < E.M * E.aslices; k += 32) avpre += st.Aval[(long long)k * W + w];
#pragma unroll
        for (int m = 0; m < PM; ++m)
            gpre[m] = (m < E.M && lane < C) ? st.gradA[((long long)m * W + w) * C + lane] : 0.0f;
    }
    if (bb0 < N) load_batch(bb0);
    if (FIN) {
        // the Jacobians of the finished evaluation and the chain-rule list go to
        // shared memory while the CV force is formed
        for (int k = threadIdx.x; k < 4 * C; k += blockDim.x) {
            Jsm[k] = st.J[(long long)w * C * 4 + k];
            acv_s[k] = __ldg(S.acv + k);
        }
        if (MODE == 1) {
            if (warp == 0) {
                const float invM = 1.0f / (float)E.M;
                // member values: lane k holds entries k and k + 32 of [M][aslices]
                const int na = E.M * E.aslices;
                float av = avpre;
                if (!pre)
                    for (int k = lane; k < na; k += 32) av += st.Aval[(long long)k * W + w];
                float d2 = 0.0f;
                for (int j = lane; j < C; j += 32) {
                    float fb = 0.0f;
                    if (pre && j == lane) {
#pragma unroll
                        for (int m = 0; m < PM; ++m)
                            if (m < E.M) fb += gpre[m];
                        fb *= invM;
#pragma unroll
                        for (int m = 0; m < PM; ++m)
                            if (m < E.M) {
                                const float d = gpre[m] - fb;
                                d2 = fmaf(d, d, d2);
                            }
                    } else {
                        for (int m = 0; m < E.M; ++m) fb += st.gradA[((long long)m * W + w) * C + j];
                        fb *= invM;
                        for (int m = 0; m < E.M; ++m) {
                            const float d = st.gradA[((long long)m * W + w) * C + j] - fb;
                            d2 = fmaf(d, d, d2);
                        }
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
                    if (p == 0) st.eps[w] = eps;
                }
            }
        } else if (MODE == 2) {
            const bool sample = KICK && t_fin >= lab.n_equil && p == 0;
            long long b = 0;
            if (sample) b = ((t_fin - lab.n_equil) * lab.B) / lab.K;
            for (int j = threadIdx.x; j < C; j += blockDim.x) {
                const long long o = (long long)w * C + j;
                const double d = rid_cv_offset(S.cv[j], (double)st.s[o], lab.s0[o]);
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
        if (slot >= 0 && p == 0) {
            if (cv_out)
                for (int j = threadIdx.x; j < C; j += blockDim.x)
                    cv_out[((long long)w * T + slot) * C + j] = st.s[(long long)w * C + j];
            if (eps_out && threadIdx.x == 0) eps_out[(long long)w * T + slot] = s_eps;
        }
    }
    double ke = 0.0;
    int bad = 0;
    for (int b0 = bb0; b0 < bb1; b0 += BATCH) {
        if (b0 > bb0) load_batch(b0);
#pragma unroll
        for (int k = 0; k < HEAD_BEADS; ++k) {
            const int i = b0 + k * HEAD_THREADS + threadIdx.x;
            if (i >= N) break;
            float4 x = make_float4(px[k].x, px[k].y, px[k].z, 0.f);
            float4 v = make_float4(pv[k].x, pv[k].y, pv[k].z, 0.f);
            float4 f = make_float4(pf[k].x, pf[k].y, pf[k].z, 0.f);
            if (FIN) {
                for (int e = a0[k]; e < a1[k]; ++e) {
                    const int2 ja = acv_s[e];
                    const float4 g = Jsm[ja.x * 4 + ja.y];
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
        if (P > 1) head_cluster_sync();   // and every slice's in its CTA
        const int cpc = (C + P - 1) / P;
        const int jend = min(C, (p + 1) * cpc);
        for (int j = p * cpc + threadIdx.x; j < jend; j += blockDim.x) {
            const int4 q = S.cv[j];
            float3 g[4];
            float sj;
            if (P == 1) {
                sj = rid_cv(q, xs, g);
            } else {
                // the CV's atoms, from the shared memory of the CTAs whose slices hold them
                const bool dist = rid_cv_is_distance(q);
                const int at[4] = {q.x, q.y, dist ? q.x : q.z, dist ? q.x : q.w};
                float4 pos[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int owner = (at[a] / BATCH) / bpc;
                    pos[a] = owner == p ? xs[at[a]] : head_ld_peer(&xs[at[a]], (uint32_t)owner);
                }
                sj = rid_cv(dist ? make_int4(0, 1, -1, -1) : make_int4(0, 1, 2, 3), pos, g);
            }
            const long long o = (long long)w * C + j;
            st.s[o] = sj;
#pragma unroll
            for (int a = 0; a < 4; ++a) st.J[o * 4 + a] = make_float4(g[a].x, g[a].y, g[a].z, 0.0f);
            float u0, u1;
            rid_cv_input(q, sj, u0, u1);
            st.u[(long long)w * 2 * C + 2 * j] = u0;
            st.u[(long long)w * 2 * C + 2 * j + 1] = u1;
        }
        if (P > 1) head_cluster_sync();   // no CTA leaves while a peer may read its positions
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
    label_stats(lab.sum + o, lab.sum2 + o, lab.bsum + o * lab.B, lab.kappa[o], lab.K, lab.B, mf[o], se[o], sd[o]);
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

__global__ void k_add_u32(uint32_t* p, uint32_t d) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *p += d;
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
    static unsigned long long attr = 0;   // positions of up to RID_MAX_BEADS beads exceed the default 48 KB
    if (rid_first_on_device(attr)) {
        cudaFuncSetAttribute(k_pair_mask, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
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

int rid_ff_default_threads(int N) { return chain_threads(N) < FF_THREADS ? chain_threads(N) : FF_THREADS; }

// CTAs per walker for W walkers and `iters` units of a walker's work (the
// force field's passes of the CTA's threads over the chain, k_head's bead
// batches): with fewer walkers than two per SM, each walker's units are split
// over up to 8 CTAs (units per CTA *ipc).  Chosen from the shape alone.
static int ff_split(int W, int iters, int& ipc) {
    static int nsm[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    int& n = nsm[dev & 63];
    if (n == 0 && cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n = 1;
    int want = (2 * n + W - 1) / (W > 0 ? W : 1);
    want = want < 1 ? 1 : (want > 8 ? 8 : want);
    if (want > iters) want = iters;
    ipc = (iters + want - 1) / want;
    return (iters + ipc - 1) / ipc;
}

// threads: CTA size (a multiple of 32 up to the default), 0 for the default.
// Each thread sums its own beads' forces in a fixed order and warps always
// cover the same 32-bead groups, so the forces do not depend on it, nor on
// the split of a walker's passes over CTAs; the energy sum does (its
// per-thread partials), so energy launches keep the default size and one CTA
// per walker.
void rid_launch_ff(const SysDev& S, StateDev st, int W, bool energy, cudaStream_t s, int threads) {
    const int dth = rid_ff_default_threads(S.N);
    const int th = (energy || threads <= 0 || threads > dth) ? dth : threads;
    const size_t sm = (size_t)rid_ff_smem_bytes(S.N);
    const bool bsm = S.N <= RID_BONDED_SMEM_MAX;
    const int iters = (S.N + th - 1) / th;
    int ipc = iters;
    const int P = energy ? 1 : ff_split(W, iters, ipc);
    static unsigned long long attr = 0;
    if (rid_first_on_device(attr)) {
        cudaFuncSetAttribute(k_ff<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_ff<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_ff<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_ff<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    }
    const unsigned grid = (unsigned)W * (unsigned)P;
    if (bsm) {
        if (energy) k_ff<true, true><<<grid, th, sm, s>>>(S, st, P, ipc);
        else k_ff<false, true><<<grid, th, sm, s>>>(S, st, P, ipc);
    } else {
        if (energy) k_ff<true, false><<<grid, th, sm, s>>>(S, st, P, ipc);
        else k_ff<false, false><<<grid, th, sm, s>>>(S, st, P, ipc);
    }
}

template <int MODE, bool FIN, bool KICK, int INT>
static void head_e(const HeadArgs& a, cudaStream_t s) {
    const int th = HEAD_THREADS;
    const size_t sm = sizeof(float4) * (size_t)a.S.N + (FIN ? (sizeof(float4) + sizeof(int2)) * 4 * (size_t)a.S.C : 0);
    static unsigned long long attr = 0;   // positions of up to RID_MAX_BEADS beads exceed the default 48 KB
    if (rid_first_on_device(attr)) {
        const int mx = (int)(sizeof(float4) * RID_MAX_BEADS + (sizeof(float4) + sizeof(int2)) * 4 * RID_MAX_CV);
        cudaFuncSetAttribute(k_head<MODE, FIN, KICK, INT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_head<MODE, FIN, KICK, INT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    }
    // CTAs per walker: a cluster over the bead batches with fewer walkers than two
    // per SM (not for energy launches, whose per-walker sums stay in one CTA, nor
    // for a server's jobs: under 16 concurrent jobs the clusters measured slower,
    // exploration p50 255 -> 281 ms on the 200/s serving stream)
    const int nb = (a.S.N + th * HEAD_BEADS - 1) / (th * HEAD_BEADS);
    int bpc = nb;
    const int P = (a.energy || INT == 0 || a.no_split) ? 1 : ff_split(a.W, nb, bpc);
    if (a.energy) {
        k_head<MODE, FIN, KICK, INT, true><<<a.W, th, sm, s>>>(a.S, a.st, a.E, a.lab, a.t_fin, a.slot, a.cv_out,
                                                                 a.eps_out, a.energy_out, a.T, a.step, 1);
    } else if (P == 1) {
        k_head<MODE, FIN, KICK, INT, false><<<a.W, th, sm, s>>>(a.S, a.st, a.E, a.lab, a.t_fin, a.slot, a.cv_out,
                                                                  a.eps_out, a.energy_out, a.T, a.step, 1);
    } else {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)(a.W * P), 1, 1);
        cfg.blockDim = dim3(th, 1, 1);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)P;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, k_head<MODE, FIN, KICK, INT, false>, a.S, a.st, a.E, a.lab, a.t_fin, a.slot,
                           a.cv_out, a.eps_out, a.energy_out, a.T, a.step, P);
    }
}

template <int MODE>
static void head_m(const HeadArgs& a, cudaStream_t s) {
    // (FIN, KICK, INT) combinations used by the host code
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

void rid_launch_add_u32(uint32_t* p, uint32_t d, cudaStream_t s) { k_add_u32<<<1, 32, 0, s>>>(p, d); }

void rid_launch_label_final(const LabelDev& lab, int W, int C, double* mf, double* se, double* sd, cudaStream_t s) {
    const long long n = (long long)W * C;
    if (n > 0) k_label_final<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(lab, W, C, mf, se, sd);
}

void rid_launch_philox(long long n, const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* words, float* normals,
                       cudaStream_t s) {
    if (n > 0) k_philox<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, ctr, k0, k1, words, normals);
}
