// rid_gemm.cuh -- the batched FP32 GEMM with fused per-pass epilogues shared
// by the training kernels (k_train.cu) and the MCMC kernels (k_mcmc.cu).
// Members of the ensemble run on grid z; activations are [M][rows][X]
// row-major.  Every output sums its K terms in increasing order.
#pragma once

#include "rid_internal.cuh"

namespace {

// Batched FP32 GEMM: C[i][j] = sum over up to two K segments of A(i, k) B(k, j)
// (member offset z * sm), so one kernel serves the N-N, N-T and T-N forms.
// Square output tiles of TS = 32 (the training GEMMs: 128-row batches, where
// small tiles are what fills the SMs) or TS = 64 (MCMC's thousands of
// walkers); K tiles of 32.  The operand tiles stream through a ring of
// shared-memory stages filled by element-wise cp.async (any strides, zero fill
// past the edges), so several tiles are in flight while one is multiplied: at
// these sizes each GEMM is bound by latency, not by its FMAs.  A 32-wide tile
// runs two K groups of 128 threads (2 x 4 outputs per thread): group q
// multiplies the K tiles q, q + 2, ... and the two partial sums are added in
// group order at the end, which halves each warp's serial chain of K tiles.
// A 64-wide tile runs one group of 256 threads (4 x 4 outputs).  Within a
// group every output sums its K terms in increasing order, so the result is
// fixed by the GEMM's shape (tile, groups) and a run is reproducible bit for
// bit.
constexpr int GK = 32;
template <int TS> struct TileCfg {
    static constexpr int groups = TS == 32 ? 2 : 1;    // K groups per CTA
    static constexpr int threads = 256;
    static constexpr int gthreads = threads / groups;  // threads of one group
    static constexpr int rp = TS * TS / gthreads / 4;  // rows per thread (4 columns each)
    static constexpr int rounds = 3;                   // rounds of `groups` K tiles in the ring
    static constexpr int stages = groups * rounds;
    static constexpr int ld = TS + 4;                  // row pitch of a stage's [GK][ld] tile
    static constexpr size_t smem = sizeof(float) * 2 * stages * GK * ld;
};

// A operand: element (i, k) at p + z sm + i si + k sk.  B operand: element
// (k, j) at p + z sm + j si + k sk (si strides the output column).
struct Operand {
    const float* p;
    long long si, sk, sm;
};
struct Seg {
    Operand a, b;
    int K;
};

enum Epi { EPI_STORE = 0, EPI_FWD = 1, EPI_BWD = 2, EPI_ADJ = 3, EPI_BACK = 4 };

// Activation tensors are [M][B][X] row-major: element (m, b, x) at
// m * B * X + b * X + x.  The epilogue pointers below follow that layout
// with the row stride ld of the GEMM's output width.
struct EpiArgs {
    float* out;        // primary output [M][rows][ld]
    long long out_sm;  // member stride of out
    int ld;            // row stride of out (= N)
    // forward: bias b_l, T_l out, h_l out, h_{l-1} in (residual), w_out (last layer: G, D out)
    const float* bias; long long bias_sm;
    float* T; float* Hout; const float* Hin; const float* wout; long long w_sm;
    float* Gout; float* Dout;
    // backward / adjoint / back: residual input, T of the layer, second outputs
    const float* res; const float* Tl; const float* Gl; float* out2; const float* tb; float* out3;
    long long act_sm;  // member stride of the [rows][ld] activations
    // dropout scales dq of the layer whose tanh the epilogue forms or reads
    // (forward, adjoint: layer l; backward, back: layer l - 1); NULL: dq = 1
    const float* Q;
    int resid;         // r_l
    int last;          // forward / adjoint on the last layer
};

struct GemmArgs {
    Seg seg[2];
    int nseg;
    int rows, cols;
    EpiArgs e;
};

// 4-byte asynchronous copy global -> shared; src_bytes = 0 writes a zero.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, int src_bytes) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may be scheduled before its predecessor on the stream has
// finished; pdl_wait() returns once the predecessor has completed and its
// memory is visible (at once for a normal launch).  pdl_trigger() lets the
// next such kernel be scheduled.  Every kernel of the chain calls pdl_wait()
// before its first memory access.  The GEMMs trigger after their K loop, so
// at most the next grid waits resident during their epilogue (a trigger at
// kernel entry let the whole chain of grids sit resident and slowed the
// training step from 244 to 327 us); the small kernels trigger at entry.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// Launch with programmatic stream serialization when pdl is set.
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
                     Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// One output tile (bx, by) of member z.
template <int EPI, int TS>
__device__ __forceinline__ void gemm_tile(const GemmArgs& g, int z, int by, int bx) {
    constexpr int NT = TileCfg<TS>::threads, RP = TileCfg<TS>::rp, NS = TileCfg<TS>::stages;
    constexpr int G = TileCfg<TS>::groups, RR = TileCfg<TS>::rounds, NTG = TileCfg<TS>::gthreads;
    constexpr int LD = TileCfg<TS>::ld;
    extern __shared__ __align__(16) float gsm[];
    float* As = gsm;                     // [NS][GK][LD]
    float* Bs = gsm + NS * GK * LD;      // [NS][GK][LD]
    const int i0 = by * TS, j0 = bx * TS;
    const int tid = threadIdx.x, grp = tid / NTG, gt = tid % NTG;
    const int tx = gt % (TS / 4), ty = gt / (TS / 4);   // rows RP ty .., columns 4 tx ..
    float acc[RP][4] = {};
    // K tiles of both segments in one sequence
    const int nt0 = (g.seg[0].K + GK - 1) / GK;
    const int nt = nt0 + (g.nseg > 1 ? (g.seg[1].K + GK - 1) / GK : 0);
    constexpr int PER = TS * GK / NT;
    // copies of K tile t into ring stage t % NS (no commit)
    auto issue_tile = [&](int t) {
        if (t >= nt) return;
        const int sidx = t < nt0 ? 0 : 1;
        const Seg& S = g.seg[sidx];
        const int k0 = (t - (sidx ? nt0 : 0)) * GK;
        const bool a_kfast = S.a.sk == 1;   // A row-major along K: threads walk K
        const bool b_jfast = S.b.si == 1;   // B (k, j) with j contiguous: threads walk j
        float* as = As + (t % NS) * GK * LD;
        float* bs = Bs + (t % NS) * GK * LD;
        const float* pa = S.a.p + (long long)z * S.a.sm;
        const float* pb = S.b.p + (long long)z * S.b.sm;
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int idx = tid + NT * r;
            const int ii = a_kfast ? idx / GK : idx % TS, kk = a_kfast ? idx % GK : idx / TS;
            const int gi = i0 + ii, gk = k0 + kk;
            const bool ia = gi < g.rows && gk < S.K;
            cp_async4(as + kk * LD + ii, ia ? pa + (long long)gi * S.a.si + (long long)gk * S.a.sk : pa, ia ? 4 : 0);
            const int jj = b_jfast ? idx % TS : idx / GK, kb = b_jfast ? idx / TS : idx % GK;
            const int gj = j0 + jj, gkb = k0 + kb;
            const bool ib = gj < g.cols && gkb < S.K;
            cp_async4(bs + kb * LD + jj, ib ? pb + (long long)gj * S.b.si + (long long)gkb * S.b.sk : pb, ib ? 4 : 0);
        }
    };
    auto mma_tile = [&](int t) {
        const float* as = As + (t % NS) * GK * LD;
        const float* bs = Bs + (t % NS) * GK * LD;
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float av[RP];
#pragma unroll
            for (int p = 0; p < RP; ++p) av[p] = as[kk * LD + ty * RP + p];
            const float4 b = *reinterpret_cast<const float4*>(&bs[kk * LD + tx * 4]);
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int p = 0; p < RP; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(av[p], bv[q], acc[p][q]);
        }
    };
    if constexpr (G == 1) {
        // one tile per ring slot: NS - 1 in flight while one is multiplied
#pragma unroll
        for (int t = 0; t < NS - 1; ++t) {
            issue_tile(t);
            cp_async_commit();             // an empty group past the end keeps the count uniform
        }
        for (int t = 0; t < nt; ++t) {
            cp_async_wait<NS - 2>();       // this thread's copies of tile t have landed
            __syncthreads();               // everyone's have, and everyone is done with tile t - 1
            issue_tile(t + NS - 1);        // refills the stage of tile t - 1
            cp_async_commit();
            mma_tile(t);
        }
        pdl_trigger();                     // the next kernel may be scheduled during the epilogue
        cp_async_wait<0>();
    } else {
        // rounds of G tiles (one per group); RR - 1 rounds in flight
        auto issue_round = [&](int R) {
#pragma unroll
            for (int q = 0; q < G; ++q) issue_tile(R * G + q);
            cp_async_commit();
        };
        const int nr = (nt + G - 1) / G;
#pragma unroll
        for (int R = 0; R < RR - 1; ++R) issue_round(R);
        for (int R = 0; R < nr; ++R) {
            cp_async_wait<RR - 2>();       // round R has landed (this thread's copies)
            __syncthreads();               // everyone's, and round R - 1 is multiplied
            issue_round(R + RR - 1);       // refills the stages of round R - 1
            if (R * G + grp < nt) mma_tile(R * G + grp);
        }
        pdl_trigger();                     // the next kernel may be scheduled during the epilogue
        cp_async_wait<0>();
        __syncthreads();                   // the ring is free: it takes the partial sums
        float* red = gsm;                  // [G - 1][TS][TS]
        if (grp > 0) {
#pragma unroll
            for (int p = 0; p < RP; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) red[((grp - 1) * TS + ty * RP + p) * TS + tx * 4 + q] = acc[p][q];
        }
        __syncthreads();
        if (grp > 0) return;               // group 0 adds the partials in group order and stores
#pragma unroll
        for (int h = 1; h < G; ++h)
#pragma unroll
            for (int p = 0; p < RP; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] += red[((h - 1) * TS + ty * RP + p) * TS + tx * 4 + q];
    }
    const EpiArgs& e = g.e;
#pragma unroll
    for (int p = 0; p < RP; ++p) {
        const int i = i0 + ty * RP + p;
        if (i >= g.rows) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + tx * 4 + q;
            if (j >= g.cols) continue;
            const long long o = (long long)z * e.act_sm + (long long)i * e.ld + j;
            const float a = acc[p][q];
            if (EPI == EPI_STORE) {
                e.out[(long long)z * e.out_sm + (long long)i * e.ld + j] = a;
            } else if (EPI == EPI_FWD) {
                // t_l = tanh(z_l); h_l = dq t_l + r h_{l-1}; last: g = w_out, d = g dq (1 - t^2)
                const float t = tanhf(a + e.bias[(long long)z * e.bias_sm + j]);
                const float dq = e.Q ? e.Q[o] : 1.0f;
                e.T[o] = t;
                if (e.Hout != e.T) e.Hout[o] = e.resid ? fmaf(dq, t, e.Hin[o]) : dq * t;
                if (e.last) {
                    const float w = e.wout[(long long)z * e.w_sm + j];
                    e.Gout[o] = w;
                    e.Dout[o] = w * (dq * (1.0f - t * t));
                }
            } else if (EPI == EPI_BWD) {
                // g_{l-1} = d_l W_l + r_l g_l; d_{l-1} = g_{l-1} dq (1 - t_{l-1}^2)
                const float gv = e.resid ? a + e.res[o] : a;
                e.out[o] = gv;
                if (e.Dout) {
                    const float t = e.Tl[o];
                    const float dq = e.Q ? e.Q[o] : 1.0f;
                    e.Dout[o] = gv * (dq * (1.0f - t * t));
                }
            } else if (EPI == EPI_ADJ) {
                // dbar = acc; gbar_l = dbar dq (1 - t^2) + r gbar_{l-1}; tbar = -2 dq t g dbar
                const float t = e.Tl[o];
                const float dq = e.Q ? e.Q[o] : 1.0f;
                const float sp = 1.0f - t * t, spq = dq * sp;
                e.out[o] = e.resid ? a * spq + e.res[o] : a * spq;
                const float tb = -2.0f * (dq * t) * e.Gl[o] * a;
                e.out2[o] = tb;
                if (e.last) e.out3[o] = tb * sp;      // zbar_{L-1} (hbar_{L-1} = 0)
            } else if (EPI == EPI_BACK) {
                // hbar_{l-1} = zbar_l W_l + r hbar_l; zbar_{l-1} = (tbar + dq hbar)(1 - t^2)
                const float hb = e.resid ? a + e.res[o] : a;
                e.out[o] = hb;
                const float t = e.Tl[o];
                const float dq = e.Q ? e.Q[o] : 1.0f;
                e.out3[o] = fmaf(dq, hb, e.tb[o]) * (1.0f - t * t);
            }
        }
    }
}


template <int EPI, int TS>
__global__ void __launch_bounds__(TileCfg<TS>::threads) k_tr_gemm(GemmArgs g) {
    pdl_wait();
    gemm_tile<EPI, TS>(g, blockIdx.z, blockIdx.y, blockIdx.x);
}

// Several independent GEMMs of one epilogue kind in one launch (grid z =
// problem x member; tiles outside a problem's extent return at once).
struct GemmBatch {
    GemmArgs g[RID_MAX_LAYERS];
    int n, M;
};
template <int EPI, int TS>
__global__ void __launch_bounds__(TileCfg<TS>::threads) k_tr_gemm_batch(GemmBatch b) {
    pdl_wait();
    const GemmArgs& g = b.g[blockIdx.z / b.M];
    if ((int)blockIdx.x * TS >= g.cols || (int)blockIdx.y * TS >= g.rows) return;
    gemm_tile<EPI, TS>(g, blockIdx.z % b.M, blockIdx.y, blockIdx.x);
}

template <int EPI, int TS>
void launch_gemm_ts(const GemmArgs& g, int M, cudaStream_t st, bool pdl) {
    static unsigned long long attr = 0;   // the ring exceeds the default 48 KB of shared memory
    if (rid_first_on_device(attr)) {
        cudaFuncSetAttribute(k_tr_gemm<EPI, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TileCfg<TS>::smem);
    }
    dim3 grid((g.cols + TS - 1) / TS, (g.rows + TS - 1) / TS, M);
    launch_k(k_tr_gemm<EPI, TS>, grid, dim3(TileCfg<TS>::threads), TileCfg<TS>::smem, st, pdl, g);
}

// pdl: launch as a programmatic dependent of the previous kernel on st.
template <int EPI>
void launch_gemm(const GemmArgs& g, int M, cudaStream_t st, bool pdl = false) {
    if (g.rows >= 1024 && g.cols >= 64)
        launch_gemm_ts<EPI, 64>(g, M, st, pdl);
    else
        launch_gemm_ts<EPI, 32>(g, M, st, pdl);
}

// The GEMMs of b (each as launch_gemm would run it with 32-wide tiles) in one launch.
template <int EPI>
void launch_gemm_batch(const GemmBatch& b, cudaStream_t st, bool pdl = false) {
    static unsigned long long attr = 0;
    if (rid_first_on_device(attr)) {
        cudaFuncSetAttribute(k_tr_gemm_batch<EPI, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TileCfg<32>::smem);
    }
    int cx = 1, cy = 1;
    for (int k = 0; k < b.n; ++k) {
        cx = (b.g[k].cols + 31) / 32 > cx ? (b.g[k].cols + 31) / 32 : cx;
        cy = (b.g[k].rows + 31) / 32 > cy ? (b.g[k].rows + 31) / 32 : cy;
    }
    launch_k(k_tr_gemm_batch<EPI, 32>, dim3(cx, cy, b.n * b.M), dim3(TileCfg<32>::threads), TileCfg<32>::smem, st,
             pdl, b);
}

// Operand helpers over [M][rows][ld] activations.
inline Operand act_rowmajor(const float* p, int ld, long long sm) { return Operand{p, (long long)ld, 1, sm}; }
inline Operand act_transposed(const float* p, int ld, long long sm) { return Operand{p, 1, (long long)ld, sm}; }

}  // namespace
