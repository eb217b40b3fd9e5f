// k_label_cons.cu -- constrained-MD labels on distance CVs (Sec. "Labeling
// phase", constrained method, Box 5: distance CVs only; Sec. "CV selection":
// the distance CV between two atoms).
//
// One CTA per run, the chain resident in shared memory for all steps.  Each
// distance CV r_j = |x_a - x_b| (distinct beads, no bead in two pairs, equal
// masses) is held at d0_j by BAOAB with SHAKE / RATTLE projections:
//   B  v += dt/2 f/m, project v
//   A  x_old = x, x += dt/2 v, SHAKE x (and v), project v
//   O  v = c1 v + c2 xi (Philox counter (bead, run, step, 0)), project v
//   A  as above;  f = force field at x;  B  v += dt/2 f/m, project v
// SHAKE for one distance: x_a -= lam r_old, x_b += lam r_old with the smaller
// root lam of |r' - 2 lam r_old| = d0 (in the cancellation-free form), and v
// changed by the same amount / h.  Projection of v: the relative velocity
// along u = (x_a - x_b) / |x_a - x_b| is removed symmetrically.
// After each step past n_equil every CV samples the mean force along its
// distance (thermodynamic integration with the r^2 Jacobian of the shell):
//   F_j = dU/dr - 2 kT / d0 = -(f_a - f_b) . u / 2 - 2 kT / d0,
// summed in FP64 with block sums for the standard error.
#include "rid_forces.cuh"

namespace {

struct ConsArgs {
    SysDev S;
    int R, C, B;
    long long n_steps, n_equil;
    uint32_t step0;
    float kT;
    const float4* x0;      // [R][N]
    const float4* v0;      // [R][N] | NULL: Maxwell-Boltzmann from Philox stream 1 at step0
    const int2* pairs;     // [C] (a, b)
    const float* d0;       // [R][C]
    double* bsum;          // [R][C][B] block sums (zeroed by the host)
    double* mf;            // [R][C]
    double* se;
    double* sd;
    float4* x_out;         // [R][N] | NULL
    float4* v_out;
    int* bad;              // [R]
};

struct ConsLayout {
    int N8, nclus;
    size_t xs, xo, vs, fs, cbox, fD, sum, sum2, bp, bytes;
};

__host__ __device__ inline ConsLayout cons_layout(int N, int C) {
    ConsLayout L{};
    L.nclus = (N + LJ_CLUSTER - 1) / LJ_CLUSTER;
    L.N8 = L.nclus * LJ_CLUSTER;
    size_t o = 0;
    L.xs = o;   o += 16 * (size_t)L.N8;
    L.xo = o;   o += 16 * (size_t)N;
    L.vs = o;   o += 16 * (size_t)N;
    L.fs = o;   o += 16 * (size_t)N;
    L.cbox = o; o += 32 * (size_t)L.nclus;
    L.sum = o;  o += 8 * (size_t)C;
    L.sum2 = o; o += 8 * (size_t)C;
    L.bp = o;   o += 8 * (size_t)C;
    L.fD = o;
    if (N <= RID_BONDED_SMEM_MAX) o += 48 * (size_t)N;
    L.bytes = (o + 15) & ~(size_t)15;
    return L;
}

constexpr int CT = 256;

// Force field (bonded + culled LJ) of every bead at xs -> fs.
__device__ void cons_forces(const SysDev& S, float4* xs, float4* cbox, float3* fD, float4* fs,
                            unsigned (*keep_s)[LJ_MAX_MASK_WORDS], bool bsm, int nclus, int& bad) {
    const int N = S.N, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwords = (nclus + 31) / 32;
    lj_cluster_boxes(xs, N, cbox);
    if (bsm)
        for (int t = tid; t < N; t += CT) bonded_dihedrals_to_smem(S, xs, t, fD);
    __syncthreads();
    const bool sig1 = S.sig2 == 1.0f;
    const float lj_s = -S.lj_eps24;
    for (int pass = 0; pass * CT < N; ++pass) {
        const int i = pass * CT + tid;
        const int wlo = i - lane, whi = wlo + 31;
        if (wlo >= N) break;                        // warp-uniform
        const bool act = i < N;
        const float3 xi = f3(xs[act ? i : N - 1]);
        lj_warp_keep_masks(S, cbox, nclus, xi, keep_s[warp]);
        const int b0 = wlo - 2 > 0 ? wlo - 2 : 0;
        const int b1 = whi + 2 < N - 1 ? whi + 2 : N - 1;
        float fx = 0.f, fy = 0.f, fz = 0.f, el = 0.f;
        if (sig1)
            lj_row_culled<true, false, true>(S, xs, cbox, keep_s[warp], nwords, xi, i, b0 / LJ_CLUSTER, b1 / LJ_CLUSTER, fx, fy,
                                       fz, el);
        else
            lj_row_culled<false, false, true>(S, xs, cbox, keep_s[warp], nwords, xi, i, b0 / LJ_CLUSTER, b1 / LJ_CLUSTER, fx, fy,
                                        fz, el);
        __syncwarp();
        if (act) {
            const float3 fb = bsm ? bonded_gather_hybrid(S, xs, i, fD) : bonded_force_on(S, xs, i);
            const float4 f = make_float4(fmaf(lj_s, fx, fb.x), fmaf(lj_s, fy, fb.y), fmaf(lj_s, fz, fb.z), 0.0f);
            bad |= !(isfinite(f.x) && isfinite(f.y) && isfinite(f.z));
            fs[i] = f;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ float3 sub3(float4 a, float4 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }

// Remove the relative velocity along each constrained pair (thread per pair).
__device__ void cons_project_v(const int2* pr, int C, const float4* xs, float4* vs) {
    for (int j = threadIdx.x; j < C; j += CT) {
        const int a = pr[j].x, b = pr[j].y;
        const float3 d = sub3(xs[a], xs[b]);
        const float ir = rsqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
        const float3 u = make_float3(d.x * ir, d.y * ir, d.z * ir);
        float4 va = vs[a], vb = vs[b];
        const float w = 0.5f * ((va.x - vb.x) * u.x + (va.y - vb.y) * u.y + (va.z - vb.z) * u.z);
        va.x -= w * u.x; va.y -= w * u.y; va.z -= w * u.z;
        vb.x += w * u.x; vb.y += w * u.y; vb.z += w * u.z;
        vs[a] = va;
        vs[b] = vb;
    }
}

// SHAKE of each pair back to d0 along its pre-step axis (thread per pair).
__device__ void cons_shake(const int2* pr, int C, const float* d0, const float4* xo, float4* xs, float4* vs, float h) {
    for (int j = threadIdx.x; j < C; j += CT) {
        const int a = pr[j].x, b = pr[j].y;
        const float3 ro = sub3(xo[a], xo[b]), rp = sub3(xs[a], xs[b]);
        const float ro2 = ro.x * ro.x + ro.y * ro.y + ro.z * ro.z;
        const float rpo = rp.x * ro.x + rp.y * ro.y + rp.z * ro.z;
        const float rp2 = rp.x * rp.x + rp.y * rp.y + rp.z * rp.z;
        const float e = rp2 - d0[j] * d0[j];
        const float dd = rpo * rpo - ro2 * e;
        const float lam = e / (2.0f * (rpo + sqrtf(dd > 0.0f ? dd : 0.0f)));
        const float ih = lam / h;
        float4 xa = xs[a], xb = xs[b], va = vs[a], vb = vs[b];
        xa.x -= lam * ro.x; xa.y -= lam * ro.y; xa.z -= lam * ro.z;
        xb.x += lam * ro.x; xb.y += lam * ro.y; xb.z += lam * ro.z;
        va.x -= ih * ro.x; va.y -= ih * ro.y; va.z -= ih * ro.z;
        vb.x += ih * ro.x; vb.y += ih * ro.y; vb.z += ih * ro.z;
        xs[a] = xa; xs[b] = xb; vs[a] = va; vs[b] = vb;
    }
}

__global__ void __launch_bounds__(CT) k_label_cons(ConsArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned keep_s[CT / 32][LJ_MAX_MASK_WORDS];
    const SysDev& S = A.S;
    const int N = S.N, C = A.C, r = blockIdx.x, tid = threadIdx.x;
    const ConsLayout L = cons_layout(N, C);
    float4* xs = reinterpret_cast<float4*>(smem + L.xs);
    float4* xo = reinterpret_cast<float4*>(smem + L.xo);
    float4* vs = reinterpret_cast<float4*>(smem + L.vs);
    float4* fs = reinterpret_cast<float4*>(smem + L.fs);
    float4* cbox = reinterpret_cast<float4*>(smem + L.cbox);
    double* sum = reinterpret_cast<double*>(smem + L.sum);
    double* sum2 = reinterpret_cast<double*>(smem + L.sum2);
    double* bp = reinterpret_cast<double*>(smem + L.bp);
    float3* fD = reinterpret_cast<float3*>(smem + L.fD);
    const bool bsm = N <= RID_BONDED_SMEM_MAX;
    const long long base = (long long)r * N;
    const float* d0 = A.d0 + (long long)r * C;
    const float kick = S.half_dt * S.inv_mass, h = S.half_dt;
    int bad = 0;

    for (int i = tid; i < L.N8; i += CT) {
        if (i < N) {
            xs[i] = A.x0[base + i];
            if (A.v0) {
                vs[i] = A.v0[base + i];
            } else {
                const float3 z = rid_normals3(rid_philox(make_uint4(i, r, A.step0, 1u), S.key0, S.key1));
                vs[i] = make_float4(S.sd_mb * z.x, S.sd_mb * z.y, S.sd_mb * z.z, 0.0f);
            }
        } else {
            xs[i] = make_float4(1.0e30f, 1.0e30f, 1.0e30f, 0.0f);
        }
    }
    for (int j = tid; j < C; j += CT) {
        sum[j] = 0.0;
        sum2[j] = 0.0;
        bp[j] = 0.0;
    }
    __syncthreads();
    // start on the constraint surface: each pair moved symmetrically along its own axis
    for (int j = tid; j < C; j += CT) {
        const int a = A.pairs[j].x, b = A.pairs[j].y;
        const float3 d = sub3(xs[a], xs[b]);
        const float s = 0.5f * d0[j] * rsqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
        const float4 pa = xs[a], pb = xs[b];
        const float3 c = make_float3(0.5f * (pa.x + pb.x), 0.5f * (pa.y + pb.y), 0.5f * (pa.z + pb.z));
        xs[a] = make_float4(c.x + s * d.x, c.y + s * d.y, c.z + s * d.z, 0.0f);
        xs[b] = make_float4(c.x - s * d.x, c.y - s * d.y, c.z - s * d.z, 0.0f);
    }
    __syncthreads();
    cons_project_v(A.pairs, C, xs, vs);
    __syncthreads();
    cons_forces(S, xs, cbox, fD, fs, keep_s, bsm, L.nclus, bad);

    const long long K = A.n_steps - A.n_equil;
    int cur_b = 0;
    auto half_drift = [&]() {
        for (int i = tid; i < N; i += CT) {
            const float4 x = xs[i], v = vs[i];
            xo[i] = x;
            xs[i] = make_float4(fmaf(h, v.x, x.x), fmaf(h, v.y, x.y), fmaf(h, v.z, x.z), 0.0f);
        }
        __syncthreads();
        cons_shake(A.pairs, C, d0, xo, xs, vs, h);
        __syncthreads();
        cons_project_v(A.pairs, C, xs, vs);
        __syncthreads();
    };
    auto half_kick = [&]() {
        for (int i = tid; i < N; i += CT) {
            float4 v = vs[i];
            const float4 f = fs[i];
            v.x = fmaf(kick, f.x, v.x);
            v.y = fmaf(kick, f.y, v.y);
            v.z = fmaf(kick, f.z, v.z);
            vs[i] = v;
        }
        __syncthreads();
        cons_project_v(A.pairs, C, xs, vs);
        __syncthreads();
    };
    for (long long t = 0; t < A.n_steps; ++t) {
        const uint32_t step = A.step0 + (uint32_t)t;
        half_kick();                                                          // B
        half_drift();                                                         // A
        if (S.c2 != 0.0f) {                                                   // O
            for (int i = tid; i < N; i += CT) {
                const float3 z = rid_normals3(rid_philox(make_uint4(i, r, step, 0u), S.key0, S.key1));
                float4 v = vs[i];
                v.x = fmaf(S.c1, v.x, S.c2 * z.x);
                v.y = fmaf(S.c1, v.y, S.c2 * z.y);
                v.z = fmaf(S.c1, v.z, S.c2 * z.z);
                vs[i] = v;
            }
            __syncthreads();
            cons_project_v(A.pairs, C, xs, vs);
            __syncthreads();
        }
        half_drift();                                                         // A
        cons_forces(S, xs, cbox, fD, fs, keep_s, bsm, L.nclus, bad);
        half_kick();                                                          // B
        if (t >= A.n_equil) {
            const long long k = t - A.n_equil;
            const int b = (int)((k * A.B) / K);
            for (int j = tid; j < C; j += CT) {
                const int pa = A.pairs[j].x, pb = A.pairs[j].y;
                const float3 d = sub3(xs[pa], xs[pb]);
                const float4 fa = fs[pa], fb = fs[pb];
                const float fu = (fa.x - fb.x) * d.x + (fa.y - fb.y) * d.y + (fa.z - fb.z) * d.z;
                const double F = -0.5 * (double)fu / (double)d0[j] - 2.0 * (double)A.kT / (double)d0[j];
                if (b != cur_b) {
                    A.bsum[((long long)r * C + j) * A.B + cur_b] = bp[j];
                    bp[j] = 0.0;
                }
                // samples enter as -F so that label_stats (-kappa mean, kappa = 1) returns mean F
                sum[j] -= F;
                sum2[j] = fma(F, F, sum2[j]);
                bp[j] -= F;
            }
            cur_b = b;
        }
    }
    __syncthreads();
    for (int j = tid; j < C; j += CT) {
        const long long o = (long long)r * C + j;
        A.bsum[o * A.B + cur_b] = bp[j];
    }
    __syncthreads();
    for (int j = tid; j < C; j += CT) {
        const long long o = (long long)r * C + j;
        double mf, se, sd;
        label_stats(&sum[j], &sum2[j], A.bsum + o * A.B, 1.0, K, A.B, mf, se, sd);
        A.mf[o] = mf;
        A.se[o] = se;
        A.sd[o] = sd;
    }
    for (int i = tid; i < N; i += CT) {
        bad |= !(isfinite(xs[i].x) && isfinite(xs[i].y) && isfinite(xs[i].z));
        if (A.x_out) A.x_out[base + i] = xs[i];
        if (A.v_out) A.v_out[base + i] = vs[i];
    }
    bad = __syncthreads_or(bad);
    if (tid == 0) A.bad[r] = bad;
}

}  // namespace

size_t rid_label_cons_smem(int N, int C) { return cons_layout(N, C).bytes; }

cudaError_t rid_launch_label_cons(const SysDev& S, int R, int C, int B, long long n_steps, long long n_equil,
                                  uint32_t step0, float kT, const float4* x0, const float4* v0, const int2* pairs,
                                  const float* d0, double* bsum, double* mf, double* se, double* sd, float4* x_out,
                                  float4* v_out, int* bad, cudaStream_t st) {
    const size_t smem = rid_label_cons_smem(S.N, C);
    cudaError_t e = cudaFuncSetAttribute(k_label_cons, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ConsArgs A{S, R, C, B, n_steps, n_equil, step0, kT, x0, v0, pairs, d0, bsum, mf, se, sd, x_out, v_out, bad};
    k_label_cons<<<R, CT, smem, st>>>(A);
    return cudaGetLastError();
}
