// k_label_fused.cu -- persistent restrained-MD kernel for batches of uneven
// label jobs (restrained method of the labeling phase).
//
// A CTA takes one (job, run) work item at a time from a global counter and
// runs all of its steps in this launch with the chain resident in shared
// memory: positions, velocities and the total force stay on chip between
// steps, so a step costs no HBM traffic besides the noise-free label sums.
// Each step applies, in the order of the per-step kernels (k_head / k_ff):
//   B A O A (Philox noise at counter (bead, run, step, 0)),
//   torsion / distance CVs and Jacobians, restraint force F_j = -kappa_j d_j
//   with d = wrap(s - s0) for a torsion and s - s0 for a distance,
//   FP64 label sample of d past n_equil,
//   force field (bonded + cluster-culled all-pairs LJ) + chain rule,
//   closing B half-kick.
// Every per-bead sum is taken in the same order as the per-step kernels, so a
// job gives the same bits here as through rid_label.
//
// Long chains run as thread-block clusters of P CTAs (CL = true): each CTA
// holds the whole chain, integrates and forms the force-field rows of its
// slice of bead passes, and sends its slice's new positions to the peers'
// shared memory (st.shared::cluster) between two cluster barriers per step;
// every CTA forms the CVs and the restraint force itself (the same
// arithmetic), CTA 0 alone keeps the label sums.  Rank 0 takes the work item
// and hands it to its peers, so a cluster leaves the loop together.
#include "rid_batch.cuh"
#include "rid_forces.cuh"

namespace {

// Shared memory carve-up for a chain of N beads and C CVs (float4 units first,
// then the FP64 label accumulators, then floats).
struct LfLayout {
    int N8, nclus;
    size_t xs, cbox, vs, fs, fD, J, dsum, dsum2, dbp, Fs, bytes;
};

__host__ __device__ inline LfLayout lf_layout(int N, int C) {
    LfLayout L{};
    L.nclus = (N + LJ_CLUSTER - 1) / LJ_CLUSTER;
    L.N8 = L.nclus * LJ_CLUSTER;
    size_t o = 0;
    L.xs = o;   o += 16 * (size_t)L.N8;
    L.cbox = o; o += 32 * (size_t)L.nclus;
    L.vs = o;   o += 16 * (size_t)N;
    L.fs = o;   o += 16 * (size_t)N;
    L.J = o;    o += 64 * (size_t)C;
    L.dsum = o; o += 8 * (size_t)C;
    L.dsum2 = o; o += 8 * (size_t)C;
    L.dbp = o;  o += 8 * (size_t)C;
    L.Fs = o;   o += 4 * (size_t)C;
    o = (o + 15) & ~(size_t)15;
    L.fD = o;
    if (N <= RID_BONDED_SMEM_MAX) o += 48 * (size_t)N;   // dihedral slots (float3 [4N])
    L.bytes = (o + 15) & ~(size_t)15;
    return L;
}

__device__ __forceinline__ uint32_t lf_peer(const void* local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(r)
                 : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(local))), "r"(rank));
    return r;
}
__device__ __forceinline__ void lf_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t lf_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Block of label sample k (of K) among B blocks.
__device__ __forceinline__ int lf_block(long long k, int B, long long K) { return (int)((k * B) / K); }

template <int NT, bool CL>
__global__ void __launch_bounds__(NT, 1024 / NT) k_label_fused(FusedArgs A, int P) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ FusedJob J;
    __shared__ int s_item;
    __shared__ unsigned keep_s[NT / 32][LJ_MAX_MASK_WORDS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rank = CL ? (int)lf_rank() : 0;
    for (;;) {
        if (tid == 0 && rank == 0) {
            const int it = atomicAdd(A.next, 1);
            s_item = it;
            if (CL)
                for (int q = 1; q < P; ++q)
                    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(lf_peer(&s_item, (uint32_t)q)), "r"(it)
                                 : "memory");
        }
        if (CL) lf_cluster_sync();
        else __syncthreads();
        if (tid == 0 && s_item < A.n_items) J = A.jobs[A.items[s_item].job];
        __syncthreads();
        const int it = s_item;
        if (it >= A.n_items) break;
        const int r = A.items[it].run;
        const SysDev& S = J.S;
        const int N = S.N, C = S.C;
        const LfLayout L = lf_layout(N, C);
        // this CTA's bead passes (all of them without a cluster)
        const int npass = (N + NT - 1) / NT, ppc = (npass + P - 1) / P;
        const int pass0 = rank * ppc, pass1 = min(npass, pass0 + ppc);
        const int lo = pass0 * NT, hi = min(N, pass1 * NT);
        float4* xs = reinterpret_cast<float4*>(smem + L.xs);
        float4* cbox = reinterpret_cast<float4*>(smem + L.cbox);
        float4* vs = reinterpret_cast<float4*>(smem + L.vs);
        float4* fs = reinterpret_cast<float4*>(smem + L.fs);
        float4* Jm = reinterpret_cast<float4*>(smem + L.J);
        double* lsum = reinterpret_cast<double*>(smem + L.dsum);
        double* lsum2 = reinterpret_cast<double*>(smem + L.dsum2);
        double* lbp = reinterpret_cast<double*>(smem + L.dbp);
        float* Fs = reinterpret_cast<float*>(smem + L.Fs);
        float3* fD = reinterpret_cast<float3*>(smem + L.fD);
        const bool bsm = N <= RID_BONDED_SMEM_MAX;
        const long long base = (long long)r * N;
        const float kick = S.half_dt * S.inv_mass;
        const float lj_s = -S.lj_eps24;
        const bool sig1 = S.sig2 == 1.0f;
        const int nwords = (L.nclus + 31) / 32;
        const long long t0 = J.t0, t1 = J.t1;
        int bad = 0;

        // ---- stage the run
        for (int i = tid; i < L.N8; i += NT) {
            if (i < N) {
                xs[i] = J.x[base + i];
                if (J.init && J.mb) {
                    const float3 z = rid_normals3(rid_philox(make_uint4(i, r, J.step0, 1u), S.key0, S.key1));
                    vs[i] = make_float4(S.sd_mb * z.x, S.sd_mb * z.y, S.sd_mb * z.z, 0.0f);
                } else {
                    vs[i] = J.v[base + i];
                }
                if (!J.init) fs[i] = J.f[base + i];
            } else {
                xs[i] = make_float4(1.0e30f, 1.0e30f, 1.0e30f, 0.0f);
            }
        }
        // label accumulators; lbp holds the partial sum of block cur_b (the block
        // of the last sample taken before this launch, else block 0)
        int cur_b = 0;
        {
            const long long kp = t0 - 1 - J.n_equil;
            if (kp >= 0) cur_b = lf_block(kp, J.B, J.K);
            for (int j = tid; j < C; j += NT) {
                const long long o = (long long)r * C + j;
                lsum[j] = J.sum[o];
                lsum2[j] = J.sum2[o];
                lbp[j] = J.bsum[o * J.B + cur_b];
            }
        }
        // (cluster: every CTA has staged the chain before any peer writes new positions into it)
        if (CL) lf_cluster_sync();
        else __syncthreads();

        // Evaluate: CVs, restraint force (and label sample at step ts >= n_equil
        // when ts >= 0), force field, chain rule; closing kick when `kick_v`.
        auto evaluate = [&](long long ts, bool kick_v) {
            lj_cluster_boxes(xs, N, cbox);
            if (bsm)
                for (int t = tid; t < N; t += NT) bonded_dihedrals_to_smem(S, xs, t, fD);
            const bool sample = ts >= J.n_equil;
            const int b = sample ? lf_block(ts - J.n_equil, J.B, J.K) : cur_b;
            const bool keep = rank == 0;   // the label sums live in CTA 0
            const bool newblock = b != cur_b;
            for (int j = tid; j < C; j += NT) {
                const int4 q = S.cv[j];
                float3 g[4];
                const float sj = rid_cv(q, xs, g);
#pragma unroll
                for (int a = 0; a < 4; ++a) Jm[4 * j + a] = make_float4(g[a].x, g[a].y, g[a].z, 0.0f);
                const long long o = (long long)r * C + j;
                const double d = rid_cv_offset(q, (double)sj, J.s0[o]);
                Fs[j] = (float)(-J.kappa[o] * d);
                if (sample && keep) {
                    if (newblock) {
                        J.bsum[o * J.B + cur_b] = lbp[j];
                        lbp[j] = 0.0;
                    }
                    lsum[j] += d;
                    lsum2[j] = fma(d, d, lsum2[j]);
                    lbp[j] += d;
                }
            }
            cur_b = b;
            __syncthreads();
            for (int pass = pass0; pass < pass1; ++pass) {
                const int i = pass * NT + tid;
                const int wlo = i - lane, whi = wlo + 31;
                if (wlo >= N) break;                        // warp-uniform
                const bool act = i < N;
                const float3 xi = f3(xs[act ? i : N - 1]);
                lj_warp_keep_masks(S, cbox, L.nclus, xi, keep_s[warp]);
                const int b0 = wlo - 2 > 0 ? wlo - 2 : 0;
                const int b1 = whi + 2 < N - 1 ? whi + 2 : N - 1;
                float fx = 0.f, fy = 0.f, fz = 0.f, el = 0.f;
                if (sig1)
                    lj_row_culled<true, false, true>(S, xs, cbox, keep_s[warp], nwords, xi, i, b0 / LJ_CLUSTER, b1 / LJ_CLUSTER,
                                               fx, fy, fz, el);
                else
                    lj_row_culled<false, false, true>(S, xs, cbox, keep_s[warp], nwords, xi, i, b0 / LJ_CLUSTER,
                                                b1 / LJ_CLUSTER, fx, fy, fz, el);
                __syncwarp();
                if (act) {
                    const float3 fb = bsm ? bonded_gather_hybrid(S, xs, i, fD) : bonded_force_on(S, xs, i);
                    float4 f = make_float4(fmaf(lj_s, fx, fb.x), fmaf(lj_s, fy, fb.y), fmaf(lj_s, fz, fb.z), 0.0f);
                    for (int e = S.acv_off[i]; e < S.acv_off[i + 1]; ++e) {
                        const int2 ja = S.acv[e];
                        const float4 g = Jm[4 * ja.x + ja.y];
                        const float fsj = Fs[ja.x];
                        f.x = fmaf(fsj, g.x, f.x);
                        f.y = fmaf(fsj, g.y, f.y);
                        f.z = fmaf(fsj, g.z, f.z);
                    }
                    bad |= !(isfinite(f.x) && isfinite(f.y) && isfinite(f.z));
                    if (kick_v) {
                        float4 v = vs[i];
                        v.x = fmaf(kick, f.x, v.x);
                        v.y = fmaf(kick, f.y, v.y);
                        v.z = fmaf(kick, f.z, v.z);
                        bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z));
                        vs[i] = v;
                    }
                    fs[i] = f;
                }
            }
            // (cluster: every CTA is done reading the positions the next step overwrites)
            if (CL) lf_cluster_sync();
            else __syncthreads();
        };

        if (J.init) evaluate(-1, false);   // force at x0 (no sample: ts = -1 < n_equil)
        for (long long t = t0; t < t1; ++t) {
            const uint32_t step = J.step0 + (uint32_t)t;
            for (int i = lo + tid; i < hi; i += NT) {
                float4 x = xs[i], v = vs[i];
                const float4 f = fs[i];
                v.x = fmaf(kick, f.x, v.x);                 // B
                v.y = fmaf(kick, f.y, v.y);
                v.z = fmaf(kick, f.z, v.z);
                x.x = fmaf(S.half_dt, v.x, x.x);            // A
                x.y = fmaf(S.half_dt, v.y, x.y);
                x.z = fmaf(S.half_dt, v.z, x.z);
                if (S.c2 != 0.0f) {                         // O
                    const float3 z = rid_normals3(rid_philox(make_uint4(i, r, step, 0u), S.key0, S.key1));
                    v.x = fmaf(S.c1, v.x, S.c2 * z.x);
                    v.y = fmaf(S.c1, v.y, S.c2 * z.y);
                    v.z = fmaf(S.c1, v.z, S.c2 * z.z);
                }
                x.x = fmaf(S.half_dt, v.x, x.x);            // A
                x.y = fmaf(S.half_dt, v.y, x.y);
                x.z = fmaf(S.half_dt, v.z, x.z);
                xs[i] = make_float4(x.x, x.y, x.z, 0.0f);
                vs[i] = v;
                if (CL)
                    for (int q = 0; q < P; ++q)
                        if (q != rank)
                            asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(
                                             lf_peer(&xs[i], (uint32_t)q)),
                                         "f"(x.x), "f"(x.y), "f"(x.z), "f"(0.0f)
                                         : "memory");
            }
            if (CL) lf_cluster_sync();   // every slice's new positions in every CTA
            else __syncthreads();
            evaluate(t, true);
        }

        // ---- write back the run (this CTA's slice; the label sums from CTA 0)
        for (int i = lo + tid; i < hi; i += NT) {
            J.x[base + i] = xs[i];
            J.v[base + i] = vs[i];
            J.f[base + i] = fs[i];
        }
        for (int j = tid; j < (rank == 0 ? C : 0); j += NT) {
            const long long o = (long long)r * C + j;
            J.sum[o] = lsum[j];
            J.sum2[o] = lsum2[j];
            J.bsum[o * J.B + cur_b] = lbp[j];
            if (t1 == J.n_steps)
                label_stats(J.sum + o, J.sum2 + o, J.bsum + o * J.B, J.kappa[o], J.K, J.B, J.mf[o], J.se[o], J.sd[o]);
        }
        bad = __syncthreads_or(bad);
        if (tid == 0 && bad) J.flags[r] = 1;
        // J and s_item are rewritten by the next item
        if (CL) lf_cluster_sync();
        else __syncthreads();
    }
}

__global__ void k_copy_descs(const CopyDesc* __restrict__ descs) {
    const CopyDesc d = descs[blockIdx.x];
    if (d.kind == 0) {
        const float* src = static_cast<const float*>(d.src);
        float4* dst = static_cast<float4*>(d.dst);
        for (long long i = threadIdx.x; i < d.n; i += blockDim.x)
            dst[i] = make_float4(src[3 * i], src[3 * i + 1], src[3 * i + 2], 0.0f);
    } else if (d.kind == 1) {
        const float4* src = static_cast<const float4*>(d.src);
        float* dst = static_cast<float*>(d.dst);
        for (long long i = threadIdx.x; i < d.n; i += blockDim.x) {
            const float4 a = src[i];
            dst[3 * i] = a.x;
            dst[3 * i + 1] = a.y;
            dst[3 * i + 2] = a.z;
        }
    } else if (d.kind == 2) {
        const double* src = static_cast<const double*>(d.src);
        double* dst = static_cast<double*>(d.dst);
        for (long long i = threadIdx.x; i < d.n; i += blockDim.x) dst[i] = src[i];
    } else if (d.kind == 3) {
        const unsigned* src = static_cast<const unsigned*>(d.src);
        unsigned* dst = static_cast<unsigned*>(d.dst);
        for (long long i = threadIdx.x; i < d.n; i += blockDim.x) dst[i] = src[i];
    } else {
        unsigned* dst = static_cast<unsigned*>(d.dst);
        for (long long i = threadIdx.x; i < d.n; i += blockDim.x) dst[i] = 0u;
    }
}

}  // namespace

void rid_launch_copy_descs(const CopyDesc* descs, int n, cudaStream_t s) {
    if (n > 0) k_copy_descs<<<n, 256, 0, s>>>(descs);
}

size_t rid_label_fused_smem(int N, int C, int threads) {
    (void)threads;
    return lf_layout(N, C).bytes;
}

template <int NT>
static cudaError_t launch_nt(const FusedArgs& A, int grid, size_t smem, int P, cudaStream_t s) {
    static unsigned long long attr = 0;
    if (rid_first_on_device(attr)) {
        cudaError_t e = cudaFuncSetAttribute(k_label_fused<NT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             220 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_label_fused<NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e != cudaSuccess) return e;
    }
    if (P <= 1) {
        k_label_fused<NT, false><<<grid, NT, smem, s>>>(A, 1);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)P;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_label_fused<NT, true>, A, P);
}

cudaError_t rid_launch_label_fused(const FusedArgs& A, int threads, int grid, size_t smem, cudaStream_t s, int cluster) {
    if (cluster > 1 && (grid % cluster || cluster > 8)) return cudaErrorInvalidValue;
    if (threads == 128) return launch_nt<128>(A, grid, smem, cluster, s);
    if (threads == 256) return launch_nt<256>(A, grid, smem, cluster, s);
    if (threads == 512) return launch_nt<512>(A, grid, smem, cluster, s);
    return cudaErrorInvalidValue;
}

int rid_label_fused_occupancy(int threads, size_t smem) {
    int n = 0;
    cudaError_t e = cudaSuccess;
    if (threads == 128) {
        cudaFuncSetAttribute(k_label_fused<128, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_label_fused<128, false>, 128, smem);
    } else if (threads == 256) {
        cudaFuncSetAttribute(k_label_fused<256, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_label_fused<256, false>, 256, smem);
    } else if (threads == 512) {
        cudaFuncSetAttribute(k_label_fused<512, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_label_fused<512, false>, 512, smem);
    }
    return e == cudaSuccess ? n : 0;
}
