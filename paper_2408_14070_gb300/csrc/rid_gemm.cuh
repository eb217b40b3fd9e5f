// rid_gemm.cuh -- the batched FP32 GEMM with fused per-pass epilogues shared
// by the training kernels (k_train.cu) and the MCMC kernels (k_mcmc.cu).
// Members of the ensemble run on grid z; activations are [M][rows][X]
// row-major.  Every output sums its K terms in increasing order.
#pragma once

#include "rid_internal.cuh"

namespace {

// Batched FP32 GEMM: C[i][j] = sum over up to two K segments of A(i, k) B(k, j)
// (member offset z * sm), so one kernel serves the N-N, N-T and T-N forms.
// Square output tiles of TS = 32 (128 threads, 2 x 4 outputs each: the
// training GEMMs have 128-row batches, and small tiles are what fills the SMs)
// or TS = 64 (256 threads, 4 x 4 outputs: MCMC's thousands of walkers); K tiles
// of 32, the next one staged in registers.  Every output sums its K terms in
// increasing order whatever the tile, so both sizes give the same bits.
constexpr int GK = 32;
template <int TS> struct TileCfg {
    static constexpr int threads = TS == 32 ? 128 : 256;
    static constexpr int rp = TS * TS / threads / 4;   // rows per thread (4 columns each)
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
    int resid;         // r_l
    int last;          // forward / adjoint on the last layer
};

struct GemmArgs {
    Seg seg[2];
    int nseg;
    int rows, cols;
    EpiArgs e;
};

__device__ __forceinline__ float ldop(const Operand& o, int z, int r, int k) {
    return o.p[(long long)z * o.sm + (long long)r * o.si + (long long)k * o.sk];
}

template <int EPI, int TS>
__global__ void __launch_bounds__(TileCfg<TS>::threads) k_tr_gemm(GemmArgs g) {
    constexpr int NT = TileCfg<TS>::threads, RP = TileCfg<TS>::rp;
    __shared__ __align__(16) float As[GK][TS + 4];
    __shared__ __align__(16) float Bs[GK][TS + 4];
    const int z = blockIdx.z, i0 = blockIdx.y * TS, j0 = blockIdx.x * TS;
    const int tid = threadIdx.x, tx = tid % (TS / 4), ty = tid / (TS / 4);   // rows RP ty .., columns 4 tx ..
    float acc[RP][4] = {};
    // K tiles of both segments in one sequence; the next tile's elements are
    // loaded into registers while the current one is multiplied
    const int nt0 = (g.seg[0].K + GK - 1) / GK;
    const int nt = nt0 + (g.nseg > 1 ? (g.seg[1].K + GK - 1) / GK : 0);
    constexpr int PER = TS * GK / NT;
    float ra[PER], rb[PER];
    auto fetch = [&](int t) {
        const int sidx = t < nt0 ? 0 : 1;
        const Seg& S = g.seg[sidx];
        const int k0 = (t - (sidx ? nt0 : 0)) * GK;
        const bool a_kfast = S.a.sk == 1;   // A row-major along K: threads walk K
        const bool b_jfast = S.b.si == 1;   // B (k, j) with j contiguous: threads walk j
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int idx = tid + NT * r;
            const int ii = a_kfast ? idx / GK : idx % TS, kk = a_kfast ? idx % GK : idx / TS;
            const int gi = i0 + ii, gk = k0 + kk;
            ra[r] = (gi < g.rows && gk < S.K) ? ldop(S.a, z, gi, gk) : 0.0f;
            const int jj = b_jfast ? idx % TS : idx / GK, kb = b_jfast ? idx / TS : idx % GK;
            const int gj = j0 + jj, gkb = k0 + kb;
            rb[r] = (gj < g.cols && gkb < S.K) ? ldop(S.b, z, gj, gkb) : 0.0f;
        }
    };
    auto stash = [&](int t) {
        const Seg& S = g.seg[t < nt0 ? 0 : 1];
        const bool a_kfast = S.a.sk == 1, b_jfast = S.b.si == 1;
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int idx = tid + NT * r;
            As[a_kfast ? idx % GK : idx / TS][a_kfast ? idx / GK : idx % TS] = ra[r];
            Bs[b_jfast ? idx / TS : idx % GK][b_jfast ? idx % TS : idx / GK] = rb[r];
        }
    };
    if (nt > 0) fetch(0);
    for (int t = 0; t < nt; ++t) {
        stash(t);
        __syncthreads();
        if (t + 1 < nt) fetch(t + 1);
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float av[RP];
#pragma unroll
            for (int p = 0; p < RP; ++p) av[p] = As[kk][ty * RP + p];
            const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int p = 0; p < RP; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(av[p], bv[q], acc[p][q]);
        }
        __syncthreads();
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
                const float t = tanhf(a + e.bias[(long long)z * e.bias_sm + j]);
                e.T[o] = t;
                if (e.Hout != e.T) e.Hout[o] = e.resid ? t + e.Hin[o] : t;
                if (e.last) {
                    const float w = e.wout[(long long)z * e.w_sm + j];
                    e.Gout[o] = w;
                    e.Dout[o] = w * (1.0f - t * t);
                }
            } else if (EPI == EPI_BWD) {
                // g_{l-1} = d_l W_l + r_l g_l; d_{l-1} = g_{l-1} (1 - t_{l-1}^2)
                const float gv = e.resid ? a + e.res[o] : a;
                e.out[o] = gv;
                if (e.Dout) {
                    const float t = e.Tl[o];
                    e.Dout[o] = gv * (1.0f - t * t);
                }
            } else if (EPI == EPI_ADJ) {
                // dbar = acc; gbar_l = dbar (1 - t^2) + r gbar_{l-1}; tbar = -2 t g dbar
                const float t = e.Tl[o];
                const float sp = 1.0f - t * t;
                e.out[o] = e.resid ? a * sp + e.res[o] : a * sp;
                const float tb = -2.0f * t * e.Gl[o] * a;
                e.out2[o] = tb;
                if (e.last) e.out3[o] = tb * sp;      // zbar_{L-1} (hbar_{L-1} = 0)
            } else if (EPI == EPI_BACK) {
                // hbar_{l-1} = zbar_l W_l + r hbar_l; zbar_{l-1} = (tbar + hbar)(1 - t^2)
                const float hb = e.resid ? a + e.res[o] : a;
                e.out[o] = hb;
                const float t = e.Tl[o];
                e.out3[o] = (e.tb[o] + hb) * (1.0f - t * t);
            }
        }
    }
}

template <int EPI>
void launch_gemm(const GemmArgs& g, int M, cudaStream_t st) {
    if (g.rows >= 1024 && g.cols >= 64) {
        dim3 grid((g.cols + 63) / 64, (g.rows + 63) / 64, M);
        k_tr_gemm<EPI, 64><<<grid, TileCfg<64>::threads, 0, st>>>(g);
    } else {
        dim3 grid((g.cols + 31) / 32, (g.rows + 31) / 32, M);
        k_tr_gemm<EPI, 32><<<grid, TileCfg<32>::threads, 0, st>>>(g);
    }
}

// Operand helpers over [M][rows][ld] activations.
inline Operand act_rowmajor(const float* p, int ld, long long sm) { return Operand{p, (long long)ld, 1, sm}; }
inline Operand act_transposed(const float* p, int ld, long long sm) { return Operand{p, 1, (long long)ld, sm}; }

}  // namespace
