// k_explore_small.cu -- every step of an exploration call for small systems
// in one persistent launch (FP32 ensembles).
//
// The per-step path launches three kernels per step (k_head, then the
// ensemble kernel beside k_ff); for a chain of a few dozen beads each of them
// runs for a few microseconds and the step is bound by launch latency.  Here
// a CTA holds one walker -- its chain, the whole FP32 ensemble, its CVs and
// Jacobians -- in shared memory and runs all steps of the call:
//   per step t: finish step t-1 (mean force, model deviation and switched
//   bias from the members' CV gradients, chain rule onto the force field,
//   closing half-kick, trace of step t-1), then B A O A with Philox noise,
//   the CVs and Jacobians at the new positions, every member's forward pass
//   and input gradient, and the force field;
// and finishes the last step at the end.  Each phase is the arithmetic of the
// per-step kernel that does it, in the same order (k_head's ensemble
// reduction and integrator, k_mlp_fp32_small's sequential dot products and
// lane-strided member value, k_ff's cluster-culled pairs with the warps on
// the same 32-bead groups), so a call gives the same bits as the per-step
// path.  Used for chains of at most 128 beads with FP32 non-residual
// ensembles of at most 8 members when the whole state fits one CTA's shared
// memory and the walkers fit one wave.
#include "rid_forces.cuh"

namespace {

constexpr int XS_THREADS = 320;   // 64 force-field threads beside 256 for the ensemble
// During a step's evaluation the force field (which needs only the new
// positions) runs on the first XS_FF threads while the ensemble (which needs
// only the CVs) runs on the rest, each group with its own named barrier.
constexpr int XS_FF = 64;
constexpr int XS_EN = XS_THREADS - XS_FF;

// acc += sum_k a[k] b[k * sb], k = 0 .. K-1 in order, the loads of 8 terms
// issued before their FMAs
__device__ __forceinline__ float xs_dot(const float* a, const float* b, int sb, int K, float acc) {
    int k = 0;
    for (; k + 8 <= K; k += 8) {
        float x[8], y[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            x[q] = a[k + q];
            y[q] = b[(k + q) * sb];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) acc = fmaf(x[q], y[q], acc);
    }
    for (; k < K; ++k) acc = fmaf(a[k], b[k * sb], acc);
    return acc;
}
__device__ __forceinline__ void xs_bar(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

struct XsArgs {
    SysDev S;
    StateDev st;
    EnsDev E;
    long long n_steps;
    uint32_t step0;
    int slot0;            // trace slot of the call's first output step
    long long T;          // trace slots of the caller's arrays
    float* cv_out;        // [W][T][C] or NULL
    float* eps_out;       // [W][T] or NULL
};

// Shared memory carve-up (bytes) for N beads, C CVs and the ensemble shape.
struct XsLayout {
    int N8, nclus;
    size_t xs, cbox, vs, fs, ff, bond, J, acv, Fs, s, u, W, b, wout, t, G0, G1, Av, gA, bytes;
};
__host__ __device__ inline int xs_wlayer(int D, int H, int l) { return l == 0 ? 0 : H * (D + 1) + (l - 1) * H * (H + 1); }
__host__ __device__ inline size_t xs_take(size_t& o, size_t n) {
    const size_t p = o;
    o = (o + n + 15) & ~(size_t)15;
    return p;
}
__host__ __device__ inline XsLayout xs_layout(int N, int C, int M, int D, int L, int H, bool bsm) {
    XsLayout Y{};
    Y.nclus = (N + LJ_CLUSTER - 1) / LJ_CLUSTER;
    Y.N8 = Y.nclus * LJ_CLUSTER;
    size_t o = 0;
    Y.xs = xs_take(o, 16 * (size_t)Y.N8);
    Y.cbox = xs_take(o, 32 * (size_t)Y.nclus);
    Y.vs = xs_take(o, 16 * (size_t)N);
    Y.fs = xs_take(o, 16 * (size_t)N);
    Y.ff = xs_take(o, 16 * (size_t)N);
    Y.bond = xs_take(o, bsm ? 12 * 8 * (size_t)N : 0);
    Y.J = xs_take(o, 16 * 4 * (size_t)C);
    Y.acv = xs_take(o, 8 * 4 * (size_t)C);
    Y.Fs = xs_take(o, 4 * (size_t)C);
    Y.s = xs_take(o, 4 * (size_t)C);
    Y.u = xs_take(o, 4 * (size_t)D);
    Y.W = xs_take(o, 4 * (size_t)xs_wlayer(D, H, L) * M);
    Y.b = xs_take(o, 4 * (size_t)M * L * H);
    Y.wout = xs_take(o, 4 * (size_t)M * H);
    Y.t = xs_take(o, 4 * (size_t)M * L * H);
    const int gw = H > D ? H : D;
    Y.G0 = xs_take(o, 4 * (size_t)M * gw);
    Y.G1 = xs_take(o, 4 * (size_t)M * gw);
    Y.Av = xs_take(o, 4 * (size_t)M);
    Y.gA = xs_take(o, 4 * (size_t)M * C);
    Y.bytes = o;
    return Y;
}

template <bool BSMEM>
__global__ void __launch_bounds__(XS_THREADS, 1) k_explore_small(XsArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned keep_s[XS_THREADS / 32][LJ_MAX_MASK_WORDS];
    __shared__ float s_eps;
    const SysDev& S = A.S;
    const EnsDev& E = A.E;
    const StateDev& st = A.st;
    const int w = blockIdx.x, N = S.N, C = S.C, W = st.W;
    const int M = E.M, D = E.D, L = E.L, H = E.H;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const XsLayout Y = xs_layout(N, C, M, D, L, H, BSMEM);
    float4* xs = reinterpret_cast<float4*>(smem + Y.xs);
    float4* cbox = reinterpret_cast<float4*>(smem + Y.cbox);
    float4* vs = reinterpret_cast<float4*>(smem + Y.vs);
    float4* fs = reinterpret_cast<float4*>(smem + Y.fs);
    float4* ff = reinterpret_cast<float4*>(smem + Y.ff);
    float3* fB = reinterpret_cast<float3*>(smem + Y.bond);   // [N] bonds, [3N] angles, [4N] dihedrals
    float3* fA = fB + N;
    float3* fD = fA + 3 * N;
    float4* Jsm = reinterpret_cast<float4*>(smem + Y.J);
    int2* acv_s = reinterpret_cast<int2*>(smem + Y.acv);
    float* Fs = reinterpret_cast<float*>(smem + Y.Fs);
    float* ss = reinterpret_cast<float*>(smem + Y.s);
    float* us = reinterpret_cast<float*>(smem + Y.u);
    float* Ws = reinterpret_cast<float*>(smem + Y.W);
    float* bs = reinterpret_cast<float*>(smem + Y.b);
    float* wo = reinterpret_cast<float*>(smem + Y.wout);
    float* ts = reinterpret_cast<float*>(smem + Y.t);
    float* G = reinterpret_cast<float*>(smem + Y.G0);
    float* Gn = reinterpret_cast<float*>(smem + Y.G1);
    float* Av = reinterpret_cast<float*>(smem + Y.Av);
    float* gA = reinterpret_cast<float*>(smem + Y.gA);
    const int wm = xs_wlayer(D, H, L);     // floats of one member's weight rows
    const int gw = H > D ? H : D;
    const long long base = (long long)w * N;
    const float kick = S.half_dt * S.inv_mass;
    const int of = S.output_freq;

    // ---- stage: the walker, the chain-rule list, the ensemble
    for (int i = tid; i < Y.N8; i += XS_THREADS) {
        if (i < N) {
            xs[i] = st.x[base + i];
            vs[i] = st.v[base + i];
            fs[i] = st.f[base + i];
        } else {
            xs[i] = make_float4(1.0e30f, 1.0e30f, 1.0e30f, 0.0f);
        }
    }
    for (int k = tid; k < 4 * C; k += XS_THREADS) acv_s[k] = __ldg(S.acv + k);
    for (int m = 0; m < M; ++m)
        for (int l = 0; l < L; ++l) {
            const int fin = l == 0 ? D : H;
            const float* Wl = E.W + (size_t)m * E.wstride + E.loff[l];
            float* dst = Ws + (size_t)m * wm + xs_wlayer(D, H, l);
            for (int idx = tid; idx < H * fin; idx += XS_THREADS) {
                const int n = idx / fin, k = idx - n * fin;
                dst[n * (fin + 1) + k] = __ldg(Wl + idx);
            }
        }
    for (int idx = tid; idx < M * L * H; idx += XS_THREADS) bs[idx] = __ldg(E.b + idx);
    for (int idx = tid; idx < M * H; idx += XS_THREADS) wo[idx] = __ldg(E.wout + idx);
    if (tid == 0) s_eps = 0.0f;
    __syncthreads();
    int bad = 0;

    // ---- finish a step (k_head's ensemble reduction): Fs = sigma(eps) * mean CV gradient,
    // trace of the finished step (its CVs, eps) into slot `slot`
    auto finish = [&](int slot) {
        if (warp == 0) {
            constexpr int PM = 8;
            const float invM = 1.0f / (float)M;
            float av = 0.0f;
            for (int k = lane; k < M; k += 32) av += Av[k];
            float gpre[PM];
#pragma unroll
            for (int m = 0; m < PM; ++m) gpre[m] = (m < M && lane < C) ? gA[m * C + lane] : 0.0f;
            float d2 = 0.0f;
            for (int j = lane; j < C; j += 32) {
                float fb = 0.0f;
                if (j == lane) {
#pragma unroll
                    for (int m = 0; m < PM; ++m)
                        if (m < M) fb += gpre[m];
                    fb *= invM;
#pragma unroll
                    for (int m = 0; m < PM; ++m)
                        if (m < M) {
                            const float d = gpre[m] - fb;
                            d2 = fmaf(d, d, d2);
                        }
                } else {
                    for (int m = 0; m < M; ++m) fb += gA[m * C + j];
                    fb *= invM;
                    for (int m = 0; m < M; ++m) {
                        const float d = gA[m * C + j] - fb;
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
            if (lane == 0) s_eps = eps;
        }
        __syncthreads();
        if (slot >= 0) {
            if (A.cv_out)
                for (int j = tid; j < C; j += XS_THREADS) A.cv_out[((long long)w * A.T + slot) * C + j] = ss[j];
            if (A.eps_out && tid == 0) A.eps_out[(long long)w * A.T + slot] = s_eps;
        }
    };

    // ---- per bead (k_head's order): with `fin`, f = fff + sum_j F_s,j ds_j/dx and the
    // closing half-kick of the finished step; with `integ`, B A O A of step `step`
    auto beads = [&](bool fin, bool integ, uint32_t step) {
        for (int i = tid; i < N; i += XS_THREADS) {
            float4 x = xs[i], v = vs[i];
            float4 f;
            if (fin) {
                const float4 g0 = ff[i];
                f = make_float4(g0.x, g0.y, g0.z, 0.f);
                const int e1 = __ldg(S.acv_off + i + 1);
                for (int e = __ldg(S.acv_off + i); e < e1; ++e) {
                    const int2 ja = acv_s[e];
                    const float4 g = Jsm[ja.x * 4 + ja.y];
                    const float fsj = Fs[ja.x];
                    f.x = fmaf(fsj, g.x, f.x);
                    f.y = fmaf(fsj, g.y, f.y);
                    f.z = fmaf(fsj, g.z, f.z);
                }
                bad |= !(isfinite(f.x) && isfinite(f.y) && isfinite(f.z));
                v.x = fmaf(kick, f.x, v.x);
                v.y = fmaf(kick, f.y, v.y);
                v.z = fmaf(kick, f.z, v.z);
                bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z));
                if (!integ) fs[i] = f;
            } else {
                const float4 g0 = fs[i];
                f = make_float4(g0.x, g0.y, g0.z, 0.f);
            }
            if (integ) {
                v.x = fmaf(kick, f.x, v.x);             // B
                v.y = fmaf(kick, f.y, v.y);
                v.z = fmaf(kick, f.z, v.z);
                x.x = fmaf(S.half_dt, v.x, x.x);        // A
                x.y = fmaf(S.half_dt, v.y, x.y);
                x.z = fmaf(S.half_dt, v.z, x.z);
                if (S.c2 != 0.0f) {                     // O
                    const float3 z = rid_normals3(rid_philox(make_uint4(i, w, step, 0u), S.key0, S.key1));
                    v.x = fmaf(S.c1, v.x, S.c2 * z.x);
                    v.y = fmaf(S.c1, v.y, S.c2 * z.y);
                    v.z = fmaf(S.c1, v.z, S.c2 * z.z);
                }
                x.x = fmaf(S.half_dt, v.x, x.x);        // A
                x.y = fmaf(S.half_dt, v.y, x.y);
                x.z = fmaf(S.half_dt, v.z, x.z);
                xs[i] = make_float4(x.x, x.y, x.z, 0.0f);
            }
            vs[i] = v;
        }
        __syncthreads();
    };

    // ---- CVs and Jacobians at the current positions, the MLP input
    auto cvs = [&]() {
        for (int j = tid; j < C; j += XS_THREADS) {
            const int4 q = S.cv[j];
            float3 g[4];
            const float sj = rid_cv(q, xs, g);
            ss[j] = sj;
#pragma unroll
            for (int a = 0; a < 4; ++a) Jsm[j * 4 + a] = make_float4(g[a].x, g[a].y, g[a].z, 0.0f);
            float u0, u1;
            rid_cv_input(q, sj, u0, u1);
            us[2 * j] = u0;
            us[2 * j + 1] = u1;
        }
        __syncthreads();
    };

    // ---- every member (k_mlp_fp32_small's arithmetic): member values, CV gradients;
    // threads XS_FF .. XS_THREADS-1
    auto ensemble = [&]() {
        const int et = tid - XS_FF, ew = et >> 5;
        for (int l = 0; l < L; ++l) {
            const int K = l == 0 ? D : H;
            for (int idx = et; idx < M * H; idx += XS_EN) {
                const int m = idx / H, n = idx - m * H;
                const float* in = l == 0 ? us : ts + ((size_t)m * L + l - 1) * H;
                const float* wr = Ws + (size_t)m * wm + xs_wlayer(D, H, l) + n * (K + 1);
                const float acc = xs_dot(in, wr, 1, K, 0.0f);
                ts[((size_t)m * L + l) * H + n] = tanhf(acc + bs[((size_t)m * L + l) * H + n]);
            }
            xs_bar(1, XS_EN);
        }
        // member value A = w_out . h_L + b_out: lane-strided partials, then the butterfly
        for (int m = ew; m < M; m += XS_EN / 32) {
            const float* hL = ts + ((size_t)m * L + L - 1) * H;
            float part = 0.0f;
            for (int n = lane; n < H; n += 32) part = fmaf(wo[m * H + n], hL[n], part);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (lane == 0) Av[m] = part + __ldg(E.bout + m);
        }
        // input gradient: g_L = w_out, Delta_l = g_l (1 - t_l^2), g_{l-1} = Delta_l W_l
        for (int idx = et; idx < M * H; idx += XS_EN) {
            const int m = idx / H, o = idx - m * H;
            G[m * gw + o] = wo[m * H + o];
        }
        xs_bar(1, XS_EN);
        for (int l = L - 1; l >= 0; --l) {
            const int Nout = l == 0 ? D : H;
            for (int idx = et; idx < M * H; idx += XS_EN) {
                const int m = idx / H, o = idx - m * H;
                const float t = ts[((size_t)m * L + l) * H + o];
                Gn[m * gw + o] = G[m * gw + o] * (1.0f - t * t);
            }
            xs_bar(1, XS_EN);
            for (int idx = et; idx < M * Nout; idx += XS_EN) {
                const int m = idx / Nout, j = idx - m * Nout;
                const float* Wl = Ws + (size_t)m * wm + xs_wlayer(D, H, l);
                G[m * gw + j] = xs_dot(Gn + m * gw, Wl + j, Nout + 1, H, 0.0f);
            }
            xs_bar(1, XS_EN);
        }
        // dA/ds_j = -sin s_j g0[2j] + cos s_j g0[2j+1] (torsion), g0[2j] (distance: input (s, 0))
        for (int idx = et; idx < M * C; idx += XS_EN) {
            const int m = idx / C, j = idx - m * C;
            const float cs = us[2 * j], sn = us[2 * j + 1];
            const float* g0 = G + m * gw;
            const bool dist = E.cvdist && __ldg(E.cvdist + j);
            gA[m * C + j] = dist ? g0[2 * j] : -sn * g0[2 * j] + cs * g0[2 * j + 1];
        }
    };

    // ---- force field (k_ff's arithmetic; warps on the same 32-bead groups); threads 0 .. XS_FF-1
    auto forcefield = [&]() {
        const int nclus = Y.nclus, nwords = (nclus + 31) / 32;
        // cluster bounding boxes (lj_cluster_boxes over this group's threads)
        for (int c = tid; c < nclus; c += XS_FF) {
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
        if (BSMEM)
            for (int t = tid; t < N; t += XS_FF) bonded_terms_to_smem(S, xs, t, fB, fA, fD);
        xs_bar(2, XS_FF);
        const bool sig1 = S.sig2 == 1.0f;
        for (int it = 0; it * XS_FF < N; ++it) {
            const int i = it * XS_FF + tid;
            const int wlo = i - lane, whi = wlo + 31;
            if (wlo >= N) break;                                  // warp-uniform
            const bool act = i < N;
            const float3 xi = f3(xs[act ? i : N - 1]);
            lj_warp_keep_masks(S, cbox, nclus, xi, keep_s[warp]);
            const int b0 = wlo - 2 > 0 ? wlo - 2 : 0;
            const int b1 = whi + 2 < N - 1 ? whi + 2 : N - 1;
            float fx = 0.f, fy = 0.f, fz = 0.f, el = 0.f;
            if (sig1)
                lj_row_culled<true, false>(S, xs, cbox, keep_s[warp], nwords, xi, i, b0 / LJ_CLUSTER, b1 / LJ_CLUSTER,
                                           fx, fy, fz, el);
            else
                lj_row_culled<false, false>(S, xs, cbox, keep_s[warp], nwords, xi, i, b0 / LJ_CLUSTER, b1 / LJ_CLUSTER,
                                            fx, fy, fz, el);
            __syncwarp();
            if (act) {
                const float3 fb = BSMEM ? bonded_gather(S, i, fB, fA, fD) : bonded_force_on(S, xs, i);
                const float sc = -S.lj_eps24;
                ff[i] = make_float4(fmaf(sc, fx, fb.x), fmaf(sc, fy, fb.y), fmaf(sc, fz, fb.z), 0.0f);
            }
        }
    };

    // ---- the call: step t finishes step t-1 (t > 0), then opens and evaluates step t
    const long long n = A.n_steps;
    auto slot_of = [&](long long t) { return ((t + 1) % of == 0) ? (int)((t + 1) / of - 1) : -1; };
    for (long long t = 0; t < n; ++t) {
        if (t > 0) finish(slot_of(t - 1));
        beads(t > 0, true, A.step0 + (uint32_t)t);
        cvs();
        if (tid < XS_FF) forcefield();   // beside the ensemble
        else ensemble();
        __syncthreads();
    }
    if (n > 0) {
        finish(slot_of(n - 1));
        beads(true, false, 0u);
    }

    // ---- write back: the state a per-step call leaves (no pending half-step)
    for (int i = tid; i < N; i += XS_THREADS) {
        st.x[base + i] = xs[i];
        st.v[base + i] = vs[i];
        st.f[base + i] = fs[i];
        st.fff[base + i] = ff[i];
    }
    for (int j = tid; j < C; j += XS_THREADS) {
        st.s[(long long)w * C + j] = ss[j];
#pragma unroll
        for (int a = 0; a < 4; ++a) st.J[((long long)w * C + j) * 4 + a] = Jsm[j * 4 + a];
        st.u[(long long)w * 2 * C + 2 * j] = us[2 * j];
        st.u[(long long)w * 2 * C + 2 * j + 1] = us[2 * j + 1];
    }
    for (int idx = tid; idx < M * C; idx += XS_THREADS) {
        const int m = idx / C, j = idx - m * C;
        st.gradA[((long long)m * W + w) * C + j] = gA[idx];
    }
    for (int m = tid; m < M; m += XS_THREADS) st.Aval[(long long)m * W + w] = Av[m];
    bad = __syncthreads_or(bad);
    if (tid == 0) {
        if (n > 0) st.eps[w] = s_eps;
        if (bad) st.flags[w] = 1;
    }
}

}  // namespace

// Shared memory of k_explore_small, or 0 when the shape is not eligible.
size_t rid_explore_small_smem(const SysDev& S, const EnsDev& E) {
    // (chains of at most 128 beads: the force field has 64 threads here, where the per-step
    // kernel splits a longer chain over several CTAs)
    if (S.N > 128 || E.resnet || E.M > 8 || E.M < 1 || S.C > 32 || E.D != 2 * S.C) return 0;
    const XsLayout Y = xs_layout(S.N, S.C, E.M, E.D, E.L, E.H, S.N <= RID_BONDED_SMEM_MAX);
    return Y.bytes <= 200 * 1024 ? Y.bytes : 0;
}

cudaError_t rid_launch_explore_small(const SysDev& S, StateDev st, const EnsDev& E, int W, long long n_steps,
                                     uint32_t step0, float* cv_out, float* eps_out, long long T, cudaStream_t s) {
    const size_t smem = rid_explore_small_smem(S, E);
    if (smem == 0) return cudaErrorInvalidValue;
    XsArgs A{};
    A.S = S;
    A.st = st;
    A.st.W = W;
    A.E = E;
    A.n_steps = n_steps;
    A.step0 = step0;
    A.T = T;
    A.cv_out = cv_out;
    A.eps_out = eps_out;
    const bool bsm = S.N <= RID_BONDED_SMEM_MAX;
    static unsigned long long attr = 0;
    if (rid_first_on_device(attr)) {
        cudaFuncSetAttribute(k_explore_small<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_explore_small<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    }
    if (bsm) k_explore_small<true><<<W, XS_THREADS, smem, s>>>(A);
    else k_explore_small<false><<<W, XS_THREADS, smem, s>>>(A);
    return cudaGetLastError();
}
