// k_mlp_fp32.cu -- plain FP32 (SIMT) ensemble MLP: forward pass and
// reverse-mode input gradient for every member on a tile of 32 walkers.
//
// Grid (ceil(W/32), M), 256 threads.  Warp w owns walkers 8 (w % 4) .. + 7
// and half (w / 4) of each block of 256 output neurons; a lane takes neurons
// n = nb + 128 (w / 4) + lane + 32 kk (kk < 4), so a thread keeps an 8 x 4
// register tile (two warps per SM sub-partition: 8 x 8 tiles on four warps
// took 261 us per step, this 238 us).  Activations live in shared memory
// transposed as [neuron][walker] rows of 36 floats (32 walkers + 4 pad:
// 16-byte aligned rows whose float4 stores by 8 consecutive lanes hit
// distinct banks).
// Weight rows (forward: W^T [in][out], backward: W [out][in], 256 output
// neurons at a time) stream from L2 into a 4-stage ring of 8 rows in shared
// memory by cp.async, so the eight warps share one copy and three stages are
// in flight while one is multiplied.  Reading every weight from L2 per warp
// (four copies, two rows in flight) took 622 us per step of 1024 walkers x
// 4 x 40-256x4-1; the ring takes 263 us.
// tanh(z_l) of every layer is kept in a global scratch [M][tile][L][32][H]
// (L2-resident at the sizes used) for the backward pass:
//   g_L = w_out,  delta_l = g_l * (1 - tanh^2 z_l),
//   g_{l-1} = W_l^T delta_l (+ g_l for a residual layer),
//   dA/ds_j = -sin s_j g_0[2j] + cos s_j g_0[2j+1].
#include "rid_internal.cuh"

namespace {

constexpr int TW = 32;    // walkers per CTA
constexpr int ROW = 36;   // shared row stride in floats
constexpr int NT = 256;   // threads per CTA: warp w takes walkers 8 (w % 4) .. and neuron half w / 4
constexpr int NK = 4;     // neuron columns per thread (of 32 lanes apart)

constexpr int KC = 8;     // weight rows per ring stage
constexpr int NSW = 4;    // ring stages
constexpr int WCOLS = 256;

__device__ __forceinline__ void cpa4(float* dst, const float* src, int bytes) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cpa16(float* dst, const float* src, int bytes) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// acc[i][kk] += sum_k in[k][8 (warp % 4) + i] * Wg[k * ldw + nb + 128 (warp / 4) + lane + 32 kk]
// The CTA's weight rows stream through a ring of NSW stages of KC rows x 256
// columns in shared memory (ws), so the eight warps share one copy; every
// accumulator still sums its K terms in increasing order.
__device__ __forceinline__ void tile_gemm(const float* __restrict__ in, int K, const float* __restrict__ Wg, int ldw,
                                          int N, int nb, int warp, int lane, float (&acc)[8][NK], float* ws) {
    const int wg = warp & 3, nh = (warp >> 2) * 32 * NK;   // walker group, neuron offset within the block
    const int nst = (K + KC - 1) / KC;
    const int ncol = N - nb < WCOLS ? N - nb : WCOLS;
    const bool vec = (ldw & 3) == 0 && (nb & 3) == 0 && (reinterpret_cast<uintptr_t>(Wg) & 15) == 0;
    auto issue = [&](int t) {
        if (t < nst) {
            float* dst = ws + (t % NSW) * KC * WCOLS;
            const int k0 = t * KC;
            if (vec) {
                for (int q = threadIdx.x; q < KC * WCOLS / 4; q += NT) {
                    const int r = q / (WCOLS / 4), c4 = 4 * (q % (WCOLS / 4)), k = k0 + r;
                    int valid = k < K ? ncol - c4 : 0;
                    valid = valid < 0 ? 0 : (valid > 4 ? 4 : valid);
                    cpa16(dst + r * WCOLS + c4, valid ? Wg + (size_t)k * ldw + nb + c4 : Wg, 4 * valid);
                }
            } else {
                for (int q = threadIdx.x; q < KC * WCOLS; q += NT) {
                    const int r = q / WCOLS, c = q % WCOLS, k = k0 + r;
                    const bool ok = k < K && c < ncol;
                    cpa4(dst + r * WCOLS + c, ok ? Wg + (size_t)k * ldw + nb + c : Wg, ok ? 4 : 0);
                }
            }
        }
        cpa_commit();
    };
#pragma unroll
    for (int t = 0; t < NSW - 1; ++t) issue(t);
    for (int t = 0; t < nst; ++t) {
        cpa_wait<NSW - 2>();
        __syncthreads();
        issue(t + NSW - 1);
        const float* wsr = ws + (t % NSW) * KC * WCOLS + nh + lane;
        const int kn = K - t * KC < KC ? K - t * KC : KC;
#pragma unroll 4
        for (int r = 0; r < kn; ++r) {
            const int k = t * KC + r;
            const float4 a0 = *reinterpret_cast<const float4*>(in + k * ROW + 8 * wg);
            const float4 a1 = *reinterpret_cast<const float4*>(in + k * ROW + 8 * wg + 4);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            float wv[NK];
#pragma unroll
            for (int kk = 0; kk < NK; ++kk) wv[kk] = wsr[r * WCOLS + 32 * kk];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int kk = 0; kk < NK; ++kk) acc[i][kk] = fmaf(a[i], wv[kk], acc[i][kk]);
        }
    }
    cpa_wait<0>();
    __syncthreads();   // the ring is refilled by the next call
}

__global__ void __launch_bounds__(NT) k_mlp_fp32(EnsDev E, StateDev st, int W, int C) {
    extern __shared__ __align__(16) float sm[];
    const int D = E.D, L = E.L, H = E.H, M = E.M;
    const int Kmax = H > D ? H : D;
    float* bufA = sm;
    float* bufB = bufA + Kmax * ROW;
    float* ubuf = bufB + Kmax * ROW;
    float* ws = ubuf + D * ROW;   // weight ring [NSW][KC][256]
    const int m = blockIdx.y, tile = blockIdx.x, ntiles = gridDim.x;
    const int w0 = tile * TW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wgp = warp & 3, nh = (warp >> 2) * 32 * NK;   // walker group, neuron offset in a block
    const float* Wm = E.W + (size_t)m * E.wstride;
    const float* WTm = E.WT + (size_t)m * E.wstride;
    float* hs = st.hs + ((size_t)m * ntiles + tile) * (size_t)L * TW * H;

    for (int idx = threadIdx.x; idx < D * TW; idx += NT) {
        const int wl = idx / D, k = idx - wl * D;
        ubuf[k * ROW + wl] = (w0 + wl < W) ? st.u[(size_t)(w0 + wl) * D + k] : 0.0f;
    }
    __syncthreads();

    // ---------------- forward
    const float* in = ubuf;
    float* out = bufA;
    for (int l = 0; l < L; ++l) {
        const int K = l == 0 ? D : H;
        const float* Wt = WTm + E.loff[l];
        const float* bias = E.b + ((size_t)m * L + l) * H;
        for (int nb = 0; nb < H; nb += 256) {
            float acc[8][NK];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int kk = 0; kk < NK; ++kk) acc[i][kk] = 0.0f;
            tile_gemm(in, K, Wt, H, H, nb, warp, lane, acc, ws);
#pragma unroll
            for (int kk = 0; kk < NK; ++kk) {
                const int n = nb + nh + lane + 32 * kk;
                if (n < H) {
                    const float bn = bias[n];
                    float h[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float t = tanhf(acc[i][kk] + bn);
                        hs[((size_t)l * TW + 8 * wgp + i) * H + n] = t;
                        h[i] = (E.resnet && l > 0) ? t + in[n * ROW + 8 * wgp + i] : t;
                    }
                    *reinterpret_cast<float4*>(out + n * ROW + 8 * wgp) = make_float4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<float4*>(out + n * ROW + 8 * wgp + 4) = make_float4(h[4], h[5], h[6], h[7]);
                }
            }
        }
        __syncthreads();
        in = out;
        out = (out == bufA) ? bufB : bufA;
    }
    // value A = w_out . h_L + b_out (warps 0-3, one per walker group)
    if (warp < 4) {
        const float* wo = E.wout + (size_t)m * H;
        float part[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int n = lane; n < H; n += 32) {
            const float wn = wo[n];
#pragma unroll
            for (int i = 0; i < 8; ++i) part[i] = fmaf(wn, in[n * ROW + 8 * warp + i], part[i]);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part[i] += __shfl_xor_sync(0xffffffffu, part[i], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int wg = w0 + 8 * warp + i;
                if (wg < W) st.Aval[(size_t)m * W + wg] = part[i] + E.bout[m];
            }
        }
    }
    // ---------------- backward: G holds g_l, Dl holds delta_l
    float* G = (in == bufA) ? bufB : bufA;   // free buffer
    float* Dl = (float*)in;                  // h_L no longer needed
    {
        const float* wo = E.wout + (size_t)m * H;
        for (int idx = threadIdx.x; idx < H * TW; idx += NT) {
            const int n = idx / TW, wl = idx - n * TW;
            G[n * ROW + wl] = wo[n];
        }
    }
    __syncthreads();
    for (int l = L - 1; l >= 0; --l) {
        const int K = H, Nout = l == 0 ? D : H;
        // delta_l = g_l * (1 - t_l^2)
        for (int idx = threadIdx.x; idx < H * TW; idx += NT) {
            const int wl = idx / H, n = idx - wl * H;
            const float t = hs[((size_t)l * TW + wl) * H + n];
            Dl[n * ROW + wl] = G[n * ROW + wl] * (1.0f - t * t);
        }
        __syncthreads();
        const float* Wl = Wm + E.loff[l];   // [H][fin] row-major = [K][Nout]
        const bool res = E.resnet && l > 0;
        float accs[8][NK];
        for (int nb = 0; nb < Nout; nb += 256) {
#pragma unroll
            for (int kk = 0; kk < NK; ++kk) {
                const int n = nb + nh + lane + 32 * kk;
#pragma unroll
                for (int i = 0; i < 8; ++i) accs[i][kk] = (res && n < Nout) ? G[n * ROW + 8 * wgp + i] : 0.0f;
            }
            tile_gemm(Dl, K, Wl, Nout, Nout, nb, warp, lane, accs, ws);
            __syncthreads();   // every thread has read G for its initial values
#pragma unroll
            for (int kk = 0; kk < NK; ++kk) {
                const int n = nb + nh + lane + 32 * kk;
                if (n < Nout) {
                    *reinterpret_cast<float4*>(G + n * ROW + 8 * wgp) =
                        make_float4(accs[0][kk], accs[1][kk], accs[2][kk], accs[3][kk]);
                    *reinterpret_cast<float4*>(G + n * ROW + 8 * wgp + 4) =
                        make_float4(accs[4][kk], accs[5][kk], accs[6][kk], accs[7][kk]);
                }
            }
        }
        __syncthreads();
    }
    // dA/ds_j = -sin s_j g0[2j] + cos s_j g0[2j+1] (torsion), g0[2j] (distance: input (s, 0))
    for (int idx = threadIdx.x; idx < C * TW; idx += NT) {
        const int wl = idx / C, j = idx - wl * C;
        const int wg = w0 + wl;
        if (wg < W) {
            const float cs = ubuf[(2 * j) * ROW + wl], sn = ubuf[(2 * j + 1) * ROW + wl];
            const bool dist = E.cvdist && __ldg(E.cvdist + j);
            const float g = dist ? G[(2 * j) * ROW + wl] : -sn * G[(2 * j) * ROW + wl] + cs * G[(2 * j + 1) * ROW + wl];
            st.gradA[((size_t)m * W + wg) * C + j] = g;
        }
    }
    (void)M;
}

// Small ensembles (every layer of a member fits in shared memory at once, as
// for widths up to about 96): one CTA per (tile of 32 walkers, member) loads
// the member's weights once -- rows of W_l [H][fin] padded to fin + 1 floats,
// so the lanes of a warp (consecutive output neurons) read distinct banks --
// and runs every layer from shared memory, with no weight ring to wait on.
// The operations are those of k_mlp_fp32 in the same order: each forward
// output is the FMA chain over its K inputs in increasing order from zero,
// then + b and tanh; each input-gradient output starts from the residual term
// (or zero) and chains over the H outputs of the layer in increasing order;
// the member value is the same lane-strided partial sums and butterfly.
constexpr int SM_MAX_FLOATS = 50 * 1024;   // 200 KB of shared memory
constexpr int SM_MAX_WIDTH = 128;          // at least two walker groups per neuron
constexpr int SR_MAX = TW / (NT / SM_MAX_WIDTH);   // walkers per thread at the widest layer: 16

struct SmallLayout {
    int woff[RID_MAX_LAYERS + 1];
    int bias, wout, u, t, h0, h1, G0, G1, total;
};
__host__ __device__ inline SmallLayout small_layout(int D, int L, int H, int resnet, int TW) {
    SmallLayout S{};
    int o = 0;
    for (int l = 0; l < L; ++l) {
        S.woff[l] = o;
        o += H * ((l == 0 ? D : H) + 1);
    }
    S.woff[L] = o;
    S.bias = o; o += L * H;
    S.wout = o; o += H;
    S.u = o;    o += TW * D;
    S.t = o;    o += L * TW * H;
    S.h0 = o;   o += resnet ? TW * H : 0;
    S.h1 = o;   o += resnet ? TW * H : 0;
    const int gw = H > D ? H : D;
    S.G0 = o;   o += TW * gw;
    S.G1 = o;   o += TW * gw;
    S.total = o;
    return S;
}

// Offset of layer l's padded weight rows (the same as SmallLayout::woff, in registers).
__device__ __forceinline__ int small_woff(int D, int H, int l) { return l == 0 ? 0 : H * (D + 1) + (l - 1) * H * (H + 1); }

// TW: walkers per CTA (1 .. 32), chosen by the launcher so that small walker
// counts still spread over many SMs; SR: a power of two bounding the walkers
// one thread carries (ceil(TW / (NT / H)) at most).
template <int SR>
__global__ void __launch_bounds__(NT) k_mlp_fp32_small(EnsDev E, StateDev st, int W, int C, int TW) {
    extern __shared__ __align__(16) float sm[];
    const int D = E.D, L = E.L, H = E.H;
    const SmallLayout Y = small_layout(D, L, H, E.resnet, TW);
    const int m = blockIdx.y, w0 = blockIdx.x * TW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float* Wm = E.W + (size_t)m * E.wstride;
    // the member's weights: every copy in flight at once, one wait
    for (int l = 0; l < L; ++l) {
        const int fin = l == 0 ? D : H;
        const float* Wl = Wm + E.loff[l];
        for (int idx = threadIdx.x; idx < H * fin; idx += NT) {
            const int n = idx / fin, k = idx - n * fin;
            cpa4(sm + small_woff(D, H, l) + n * (fin + 1) + k, Wl + idx, 4);
        }
    }
    cpa_commit();
    for (int idx = threadIdx.x; idx < L * H; idx += NT) sm[Y.bias + idx] = __ldg(E.b + (size_t)m * L * H + idx);
    for (int idx = threadIdx.x; idx < H; idx += NT) sm[Y.wout + idx] = __ldg(E.wout + (size_t)m * H + idx);
    for (int idx = threadIdx.x; idx < TW * D; idx += NT) {
        const int wl = idx / D, k = idx - wl * D;
        sm[Y.u + idx] = (w0 + wl < W) ? st.u[(size_t)(w0 + wl) * D + k] : 0.0f;
    }
    cpa_wait<0>();
    __syncthreads();
    // forward: t_l = tanh(in W_l^T + b_l), h_l = t_l (+ h_{l-1} for a residual layer)
    const float* in = sm + Y.u;
    for (int l = 0; l < L; ++l) {
        const int K = l == 0 ? D : H;
        const float* Wl = sm + small_woff(D, H, l);
        float* tl = sm + Y.t + l * TW * H;
        const bool res = E.resnet && l > 0;
        float* hout = E.resnet ? sm + ((l & 1) ? Y.h1 : Y.h0) : tl;
        // thread -> neuron n and walkers g, g + P, ...: one weight read per k
        // serves SR independent chains
        const int P = NT / H, n = threadIdx.x % H, g = threadIdx.x / H;
        if (g < P) {
            float acc[SR];
#pragma unroll
            for (int r = 0; r < SR; ++r) acc[r] = 0.0f;
            const float* wr = Wl + n * (K + 1);
            for (int k = 0; k < K; ++k) {
                const float wv = wr[k];
#pragma unroll
                for (int r = 0; r < SR; ++r)
                    if (g + P * r < TW) acc[r] = fmaf(in[(g + P * r) * K + k], wv, acc[r]);
            }
            const float bn = sm[Y.bias + l * H + n];
#pragma unroll
            for (int r = 0; r < SR; ++r) {
                const int wl = g + P * r;
                if (wl < TW) {
                    const float t = tanhf(acc[r] + bn);
                    tl[wl * H + n] = t;
                    if (E.resnet) hout[wl * H + n] = res ? t + in[wl * K + n] : t;
                }
            }
        }
        __syncthreads();
        in = hout;
    }
    // member value A = w_out . h_L + b_out: lane-strided partials, then the butterfly
    for (int wl = warp; wl < TW; wl += NT / 32) {
        float part = 0.0f;
        for (int n = lane; n < H; n += 32) part = fmaf(sm[Y.wout + n], in[wl * H + n], part);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0 && w0 + wl < W) st.Aval[(size_t)m * W + w0 + wl] = part + E.bout[m];
    }
    // input gradient: g_L = w_out, Delta_l = g_l (1 - t_l^2), g_{l-1} = Delta_l W_l (+ g_l)
    float* G = sm + Y.G0;
    float* Gn = sm + Y.G1;
    for (int o = threadIdx.x; o < TW * H; o += NT) G[o] = sm[Y.wout + (o % H)];
    __syncthreads();
    for (int l = L - 1; l >= 0; --l) {
        const int Nout = l == 0 ? D : H, fin = Nout;
        const float* tl = sm + Y.t + l * TW * H;
        const float* Wl = sm + small_woff(D, H, l);
        const bool res = E.resnet && l > 0;
        float* Dl = Gn;   // Delta_l in the free buffer, then g_{l-1} over G
        for (int o = threadIdx.x; o < TW * H; o += NT) {
            const float t = tl[o];
            Dl[o] = G[o] * (1.0f - t * t);
        }
        __syncthreads();
        // g_{l-1}[j] = (g_l[j] if residual) + sum_k Delta_l[k] W_l[k][j], written over G after all reads
        // thread -> input j and walkers g, g + P, ... (P = NT / Nout groups, at most TW)
        {
            const int P = NT / Nout < TW ? NT / Nout : TW, j = threadIdx.x % Nout, g = threadIdx.x / Nout;
            float acc[SR];
            const bool act = g < P;
#pragma unroll
            for (int r = 0; r < SR; ++r) {
                const int wl = g + P * r;
                acc[r] = (act && wl < TW && res) ? G[wl * H + j] : 0.0f;
            }
            if (act)
                for (int k = 0; k < H; ++k) {
                    const float wv = Wl[k * (fin + 1) + j];
#pragma unroll
                    for (int r = 0; r < SR; ++r)
                        if (g + P * r < TW) acc[r] = fmaf(Dl[(g + P * r) * H + k], wv, acc[r]);
                }
            __syncthreads();   // every thread has read G for its initial values
            if (act)
#pragma unroll
                for (int r = 0; r < SR; ++r) {
                    const int wl = g + P * r;
                    if (wl < TW) G[wl * (l == 0 ? D : H) + j] = acc[r];
                }
            __syncthreads();
        }
    }
    // dA/ds_j = -sin s_j g0[2j] + cos s_j g0[2j+1] (torsion), g0[2j] (distance: input (s, 0))
    for (int idx = threadIdx.x; idx < C * TW; idx += NT) {
        const int wl = idx / C, j = idx - wl * C;
        const int wg = w0 + wl;
        if (wg < W) {
            const float cs = sm[Y.u + wl * D + 2 * j], sn = sm[Y.u + wl * D + 2 * j + 1];
            const float* g0 = G + wl * D;
            const bool dist = E.cvdist && __ldg(E.cvdist + j);
            st.gradA[((size_t)m * W + wg) * C + j] = dist ? g0[2 * j] : -sn * g0[2 * j] + cs * g0[2 * j + 1];
        }
    }
}

}  // namespace

size_t rid_mlp_fp32_scratch_floats(int W, int M, int L, int H) {
    const size_t ntiles = (size_t)(W + TW - 1) / TW;
    return (size_t)M * ntiles * L * TW * H;
}

void rid_launch_mlp_fp32(const EnsDev& E, StateDev st, int W, int C, cudaStream_t s) {
    // walkers per CTA: the largest power of two up to 32 that still gives one
    // wave of CTAs (152 SMs), at least one walker
    int tw = 32;
    while (tw > 1 && (long long)((W + tw - 1) / tw) * E.M < 152) tw >>= 1;
    const SmallLayout Y = small_layout(E.D, E.L, E.H, E.resnet, tw);
    if (Y.total <= SM_MAX_FLOATS && small_layout(E.D, E.L, E.H, E.resnet, 32).total <= SM_MAX_FLOATS &&
        E.H <= SM_MAX_WIDTH && E.D <= NT) {
        const int wpt = (tw + NT / E.H - 1) / (NT / E.H);
        int sr = 1;
        while (sr < wpt) sr <<= 1;
        auto kern = sr == 1 ? k_mlp_fp32_small<1> : sr == 2 ? k_mlp_fp32_small<2> : sr == 4 ? k_mlp_fp32_small<4>
                  : sr == 8 ? k_mlp_fp32_small<8> : k_mlp_fp32_small<SR_MAX>;
        static unsigned long long attr_small = 0;
        if (rid_first_on_device(attr_small))
            for (auto k : {k_mlp_fp32_small<1>, k_mlp_fp32_small<2>, k_mlp_fp32_small<4>, k_mlp_fp32_small<8>,
                           k_mlp_fp32_small<SR_MAX>})
                cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_MAX_FLOATS * 4);
        kern<<<dim3((W + tw - 1) / tw, E.M), NT, (size_t)Y.total * sizeof(float), s>>>(E, st, W, C, tw);
        return;
    }
    const int Kmax = E.H > E.D ? E.H : E.D;
    const size_t sm = sizeof(float) * ((size_t)2 * Kmax * ROW + (size_t)E.D * ROW + (size_t)NSW * KC * WCOLS);
    static unsigned long long attr_set = 0;
    if (rid_first_on_device(attr_set)) {
        // activations 2 x 512 x 36 + inputs 256 x 36 + ring 4 x 8 x 256 floats = 212 KB at the limits
        cudaFuncSetAttribute(k_mlp_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    }
    dim3 grid((W + TW - 1) / TW, E.M);
    k_mlp_fp32<<<grid, NT, sm, s>>>(E, st, W, C);
}
