// k_noalloc.cu -- ensemble member gradients without any device allocation.
//
// For callers that cannot allocate device memory themselves or through the
// library -- a host framework that hands out all device memory from its own
// pool (an allocation behind its back escapes its accounting and fails once
// the pool has reserved the device), or an embedding that forbids allocation
// after start-up (cudaMalloc can synchronise the device and take unbounded
// time) -- rid_ensemble_grad_noalloc evaluates the ensemble on caller-given
// CV points with caller-given device arrays only.  The one piece of scratch the
// computation needs -- the tanh activations of every hidden layer, kept for
// the reverse pass -- lives in a file-scope static device array of fixed size
// that every GPU loading this library holds until the process exits.
//
// The arithmetic is the FP32 SIMT ensemble kernel's (same tiles, same
// summation order), reading the weights straight from the packed model layout
// instead of the library's transposed device copies.  That costs speed in the
// forward pass: the lanes of a warp read weights of different output units,
// K floats apart, so every weight load touches 32 sectors; the entry point is
// therefore several times slower than the ensemble stage of rid_eval_forces.
#include <mutex>

#include "rid_internal.cuh"

// 2 Mi floats = 8 MiB of activation scratch per device: e.g. 1024 points x
// 4 members x 4 layers x width 128, or 512 points x 4 x 4 x 256.
#define RID_NOALLOC_SCRATCH_FLOATS (2u * 1024u * 1024u)
#define RID_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) float g_noalloc_scratch[RID_NOALLOC_SCRATCH_FLOATS];

namespace {

constexpr int TW = 32;    // CV points per CTA
constexpr int ROW = 36;   // shared row stride in floats
constexpr int NT = 128;   // threads per CTA
// Largest dynamic shared memory: 2 max(H, D) + D rows of 36 floats with
// H <= 512 and D <= 256.
constexpr int NOALLOC_SMEM_MAX = (2 * 512 + 256) * ROW * 4;

struct PackedNet {
    const float* w;       // [M][P] packed: W_1[H][D], b_1, (W_l[H][H], b_l) l=2..L, w_out[H], b_out
    long long P;          // floats per model
    long long woff[RID_MAX_LAYERS];   // offset of W_l within a model
    long long boff[RID_MAX_LAYERS];   // offset of b_l
    long long ooff;                   // offset of w_out (b_out follows)
    int M, D, L, H, resnet;
};

// acc[i][kk] += sum_k in[k][8 warp + i] * Wg[k * sk + (nb + lane + 32 kk) * sn]
__device__ __forceinline__ void tile_gemm_strided(const float* __restrict__ in, int K, const float* __restrict__ Wg,
                                                  long long sk, long long sn, int N, int nb, int warp, int lane,
                                                  float (&acc)[8][8]) {
    bool ok[8];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) ok[kk] = nb + lane + 32 * kk < N;
#pragma unroll 2
    for (int k = 0; k < K; ++k) {
        const float4 a0 = *reinterpret_cast<const float4*>(in + k * ROW + 8 * warp);
        const float4 a1 = *reinterpret_cast<const float4*>(in + k * ROW + 8 * warp + 4);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        float wv[8];
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
            wv[kk] = ok[kk] ? __ldg(Wg + (long long)k * sk + (long long)(nb + lane + 32 * kk) * sn) : 0.0f;
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) acc[i][kk] = fmaf(a[i], wv[kk], acc[i][kk]);
    }
}

// Grid (ceil(W/32), M), 128 threads; hs = the static scratch.
__global__ void __launch_bounds__(NT) k_mlp_noalloc(PackedNet E, const float* __restrict__ s, int W, int C,
                                                    float* __restrict__ hs, float* __restrict__ gradA,
                                                    float* __restrict__ Aval) {
    extern __shared__ __align__(16) float sm[];
    const int D = E.D, L = E.L, H = E.H;
    const int Kmax = H > D ? H : D;
    float* bufA = sm;
    float* bufB = bufA + Kmax * ROW;
    float* ubuf = bufB + Kmax * ROW;
    const int m = blockIdx.y, tile = blockIdx.x, ntiles = gridDim.x;
    const int w0 = tile * TW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float* wm = E.w + (size_t)m * E.P;
    float* hst = hs + ((size_t)m * ntiles + tile) * (size_t)L * TW * H;

    // input u = (cos s_j, sin s_j)
    for (int idx = threadIdx.x; idx < C * TW; idx += NT) {
        const int wl = idx / C, j = idx - wl * C;
        float sn = 0.0f, cs = 0.0f;
        if (w0 + wl < W) sincosf(s[(size_t)(w0 + wl) * C + j], &sn, &cs);
        ubuf[(2 * j) * ROW + wl] = cs;
        ubuf[(2 * j + 1) * ROW + wl] = sn;
    }
    __syncthreads();

    const float* in = ubuf;
    float* out = bufA;
    for (int l = 0; l < L; ++l) {
        const int K = l == 0 ? D : H;
        const float* Wl = wm + E.woff[l];     // [H][K] row-major: element (k, n) at n K + k
        const float* bias = wm + E.boff[l];
        for (int nb = 0; nb < H; nb += 256) {
            float acc[8][8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) acc[i][kk] = 0.0f;
            tile_gemm_strided(in, K, Wl, 1, K, H, nb, warp, lane, acc);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const int n = nb + lane + 32 * kk;
                if (n < H) {
                    const float bn = bias[n];
                    float h[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float t = tanhf(acc[i][kk] + bn);
                        hst[((size_t)l * TW + 8 * warp + i) * H + n] = t;
                        h[i] = (E.resnet && l > 0) ? t + in[n * ROW + 8 * warp + i] : t;
                    }
                    *reinterpret_cast<float4*>(out + n * ROW + 8 * warp) = make_float4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<float4*>(out + n * ROW + 8 * warp + 4) = make_float4(h[4], h[5], h[6], h[7]);
                }
            }
        }
        __syncthreads();
        in = out;
        out = (out == bufA) ? bufB : bufA;
    }
    // value A = w_out . h_L + b_out
    {
        const float* wo = wm + E.ooff;
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
        if (lane == 0 && Aval) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int wg = w0 + 8 * warp + i;
                if (wg < W) Aval[(size_t)m * W + wg] = part[i] + wo[H];
            }
        }
    }
    // reverse pass: G holds g_l, Dl holds delta_l
    float* G = (in == bufA) ? bufB : bufA;
    float* Dl = (float*)in;
    {
        const float* wo = wm + E.ooff;
        for (int idx = threadIdx.x; idx < H * TW; idx += NT) {
            const int n = idx / TW, wl = idx - n * TW;
            G[n * ROW + wl] = wo[n];
        }
    }
    __syncthreads();
    for (int l = L - 1; l >= 0; --l) {
        const int K = H, Nout = l == 0 ? D : H;
        for (int idx = threadIdx.x; idx < H * TW; idx += NT) {
            const int wl = idx / H, n = idx - wl * H;
            const float t = hst[((size_t)l * TW + wl) * H + n];
            Dl[n * ROW + wl] = G[n * ROW + wl] * (1.0f - t * t);
        }
        __syncthreads();
        const float* Wl = wm + E.woff[l];     // [H][Nout] row-major = [K][N]
        const bool res = E.resnet && l > 0;   // g_{l-1} = W_l^T delta_l + g_l
        float accs[8][8];
        for (int nb = 0; nb < Nout; nb += 256) {
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const int n = nb + lane + 32 * kk;
#pragma unroll
                for (int i = 0; i < 8; ++i) accs[i][kk] = (res && n < Nout) ? G[n * ROW + 8 * warp + i] : 0.0f;
            }
            tile_gemm_strided(Dl, K, Wl, Nout, 1, Nout, nb, warp, lane, accs);
            __syncthreads();   // every thread has read G before it is overwritten
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const int n = nb + lane + 32 * kk;
                if (n < Nout) {
                    *reinterpret_cast<float4*>(G + n * ROW + 8 * warp) =
                        make_float4(accs[0][kk], accs[1][kk], accs[2][kk], accs[3][kk]);
                    *reinterpret_cast<float4*>(G + n * ROW + 8 * warp + 4) =
                        make_float4(accs[4][kk], accs[5][kk], accs[6][kk], accs[7][kk]);
                }
            }
        }
        __syncthreads();
    }
    // dA/ds_j = -sin s_j g0[2j] + cos s_j g0[2j+1]
    for (int idx = threadIdx.x; idx < C * TW; idx += NT) {
        const int wl = idx / C, j = idx - wl * C;
        const int wg = w0 + wl;
        if (wg < W) {
            const float cs = ubuf[(2 * j) * ROW + wl], sn = ubuf[(2 * j + 1) * ROW + wl];
            gradA[((size_t)m * W + wg) * C + j] = -sn * G[(2 * j) * ROW + wl] + cs * G[(2 * j + 1) * ROW + wl];
        }
    }
}

// Device address of the static scratch, looked up once per device (the first
// call on a device does it, under a lock).
std::mutex g_mu;
float* g_scratch_ptr[RID_NOALLOC_MAX_DEVICES] = {nullptr};

}  // namespace

extern "C" int rid_ensemble_grad_noalloc(int32_t n_points, int32_t n_cv, const float* s, int32_t n_models,
                                         int32_t n_layers, int32_t width, int32_t resnet, const float* weights,
                                         float* grad_out, float* value_out, void* stream) {
    NvtxScope nvtx_("rid_ensemble_grad_noalloc");
    const int W = n_points, C = n_cv, M = n_models, L = n_layers, H = width, D = 2 * n_cv;
    if (!s || !weights || !grad_out) return rid_fail(RID_ERR_ARG, "rid_ensemble_grad_noalloc: NULL array argument");
    if (W < 1 || C < 1 || C > RID_MAX_CV || M < 1 || M > RID_MAX_MODELS || L < 1 || L > RID_MAX_LAYERS || H < 32 ||
        H > RID_MAX_WIDTH || H % 32 || (resnet != 0 && resnet != 1))
        return rid_fail(RID_ERR_ARG,
                        "rid_ensemble_grad_noalloc: need n_points >= 1, 1 <= n_cv <= %d, 1 <= n_models <= %d, "
                        "1 <= n_layers <= %d, width a multiple of 32 in [32, %d], resnet 0 or 1",
                        RID_MAX_CV, RID_MAX_MODELS, RID_MAX_LAYERS, RID_MAX_WIDTH);
    const size_t ntiles = (size_t)(W + TW - 1) / TW;
    const size_t need = (size_t)M * ntiles * L * TW * H;
    if (need > RID_NOALLOC_SCRATCH_FLOATS)
        return rid_fail(RID_ERR_ARG,
                        "rid_ensemble_grad_noalloc: scratch n_models * ceil(n_points/32) * 32 * n_layers * width = "
                        "%zu floats exceeds the fixed %u floats (8 MiB)",
                        need, (unsigned)RID_NOALLOC_SCRATCH_FLOATS);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return rid_fail(RID_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= RID_NOALLOC_MAX_DEVICES)
        return rid_fail(RID_ERR_ARG, "rid_ensemble_grad_noalloc: device ordinal %d >= %d", dev, RID_NOALLOC_MAX_DEVICES);
    float* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return rid_fail(RID_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            e = cudaFuncSetAttribute(k_mlp_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize, NOALLOC_SMEM_MAX);
            if (e != cudaSuccess) return rid_fail(RID_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
            g_scratch_ptr[dev] = static_cast<float*>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    PackedNet E{};
    E.w = weights;
    E.M = M; E.D = D; E.L = L; E.H = H; E.resnet = resnet;
    long long off = 0;
    for (int l = 0; l < L; ++l) {
        E.woff[l] = off;
        off += (long long)H * (l == 0 ? D : H);
        E.boff[l] = off;
        off += H;
    }
    E.ooff = off;
    E.P = off + H + 1;
    const int Kmax = H > D ? H : D;
    const size_t smem = sizeof(float) * ((size_t)2 * Kmax * ROW + (size_t)D * ROW);
    k_mlp_noalloc<<<dim3((unsigned)ntiles, (unsigned)M), NT, smem, (cudaStream_t)stream>>>(E, s, W, C, scratch,
                                                                                          grad_out, value_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return rid_fail(RID_ERR_CUDA, "k_mlp_noalloc launch: %s", cudaGetErrorString(e));
    return RID_OK;
}
