// k_train.cu -- training the ensemble on mean-force labels (Sec. "Training
// phase": numb_models, neurons, resnet, batch_size, init_lr, decay_steps,
// decay_rate; Sec. "Training": the models are fitted to the labelled mean
// forces, the derivatives of the free energy).
//
// Each member i is fitted on its own batches: the loss is the mean squared
// difference between its CV gradient dA_i/ds and the label MF over the batch
// and the C components, and the weights take one Adam step per batch with the
// learning rate init_lr * decay_rate^(t / decay_steps).
//
// One training step is a chain of batched FP32 GEMMs (members on grid z) with
// the elementwise work of each pass fused into the GEMM that produces its
// input (notation of the per-layer recurrences; r_l = 1 for residual layers):
//   forward    l = 0..L-1:  t_l = tanh(h_{l-1} W_l^T + b_l), h_l = t_l + r_l h_{l-1}
//                           (last layer: g_{L-1} = w_out, d_{L-1} = g (1 - t^2))
//   input grad l = L-1..0:  g_{l-1} = d_l W_l + r_l g_l, d_{l-1} = g_{l-1} (1 - t_{l-1}^2)
//   loss:                   dA/ds_j = -sin s_j g[2j] + cos s_j g[2j+1], its adjoint gbar_{-1}
//   adjoint    l = 0..L-1:  dbar = gbar_{l-1} W_l^T, gbar_l = dbar (1 - t^2) + r_l gbar_{l-1},
//                           tbar_l = -2 t_l g_l dbar  (last layer: zbar = tbar (1 - t^2))
//   back       l = L-1..1:  hbar_{l-1} = zbar_l W_l + r_l hbar_l,
//                           zbar_{l-1} = (tbar_{l-1} + hbar_{l-1}) (1 - t_{l-1}^2)
//   weights:   dW_l = d_l^T gbar_{l-1} + zbar_l^T h_{l-1} (one GEMM over 2B rows),
//              db_l = sum_b zbar_l, dw_out = sum_b gbar_{L-1}, db_out = 0
//   Adam (Kingma & Ba) on every parameter.
// Dropout (drop_out_rate) scales each hidden unit's tanh by q in {0, 1/(1-p)}:
// h_l = q t_l + r_l h_{l-1}, and every (1 - t^2) above that belongs to a
// layer's activation derivative becomes q (1 - t^2), tbar_l gains the factor
// q, and zbar_{l-1} = (tbar + q hbar)(1 - t^2).  The masks come from Philox,
// one counter per four units, drawn by the batch gather of each step.
// Every sum is taken in a fixed order, so a run is reproducible bit for bit.
#include <cmath>
#include <vector>

#include "rid_gemm.cuh"

namespace {

// Dropout scales of one step (one Philox block per four units):
// Q[l][m][b][j] = 1/(1-p) iff word j % 4 of Philox(j / 4 + nw (l + L m), b,
// step, 4) >= thr, else 0 (nw = ceil(H / 4)).
struct MaskArgs {
    float* Q;                  // NULL: no dropout
    int L, H;
    uint32_t step, thr, k0, k1;
    float scale;
};
__device__ __forceinline__ void tr_mask_block(const MaskArgs& a, int M, int B, long long e) {
    const int nw = (a.H + 3) / 4;
    const int k = (int)(e % nw);
    const long long r = e / nw;                       // (l, m, b)
    const int b = (int)(r % B);
    const long long lm = r / B;                       // l M + m
    const int m = (int)(lm % M), l = (int)(lm / M);
    const uint4 x = rid_philox(make_uint4((uint32_t)(k + nw * (l + a.L * m)), (uint32_t)b, a.step, 4u), a.k0, a.k1);
    const uint32_t wd[4] = {x.x, x.y, x.z, x.w};
    float* q = a.Q + r * a.H + 4 * k;
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (4 * k + c < a.H) q[c] = wd[c] >= a.thr ? a.scale : 0.0f;
}

// u = (cos s, sin s) of each member's batch ((s, 0) for a distance CV:
// dist[j] != 0), plus the batch's s and labels, and the step's dropout
// scales.  idx is checked; an index outside [0, n) reads sample 0 and sets *bad.
__global__ void k_tr_gather(const int* __restrict__ idx, const float* __restrict__ s, const float* __restrict__ mf,
                            int n, int M, int B, int C, float* __restrict__ U, float* __restrict__ SB,
                            float* __restrict__ MFB, int* bad, MaskArgs mk, const int* __restrict__ dist) {
    pdl_trigger();
    pdl_wait();
    if (mk.Q) {
        const long long nm = (long long)mk.L * M * B * ((mk.H + 3) / 4);
        for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nm; e += (long long)gridDim.x * blockDim.x)
            tr_mask_block(mk, M, B, e);
    }
    const long long tot = (long long)M * B * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long mb = e / C;
        const int j = (int)(e - mb * C);
        int k = idx[mb];
        if (k < 0 || k >= n) {
            atomicOr(bad, 1);
            k = 0;
        }
        const float sv = s[(long long)k * C + j];
        if (dist && dist[j]) {
            U[mb * 2 * C + 2 * j] = sv;
            U[mb * 2 * C + 2 * j + 1] = 0.0f;
        } else {
            float sn, cs;
            sincosf(sv, &sn, &cs);
            U[mb * 2 * C + 2 * j] = cs;
            U[mb * 2 * C + 2 * j + 1] = sn;
        }
        SB[e] = sv;
        MFB[e] = mf[(long long)k * C + j];
    }
}

// Per member (grid y) and chunk of LT (sample, CV) pairs (grid x): residual
// dA/ds - MF, gbar_{-1} = d loss / d(dA/du), and the chunk's sum of squared
// residuals (a fixed-order tree) into lpart[m][chunk]; k_tr_colsum adds the
// chunks in order into the loss.
constexpr int LT = 256;
__global__ void __launch_bounds__(LT) k_tr_loss(const float* __restrict__ G0, const float* __restrict__ SB,
                                                const float* __restrict__ MFB, int B, int C,
                                                float* __restrict__ GB0, double* __restrict__ lpart,
                                                const int* __restrict__ dist) {
    pdl_trigger();
    pdl_wait();
    __shared__ double red[LT];
    const int m = blockIdx.y;
    const long long n = (long long)B * C;
    const float scale = 2.0f / (float)n;
    double part = 0.0;
    const long long e = (long long)blockIdx.x * LT + threadIdx.x;
    if (e < n) {
        const long long o = (long long)m * n + e;
        const float sv = SB[o];
        const long long u = (long long)m * 2 * n + 2 * e;     // (b, j) -> u index 2 (b C + j)
        // a distance CV (input (s, 0)): dA/ds = dA/du_2j; a torsion: through (cos, sin)
        const bool dj = dist && dist[e % C];
        float sn = 0.0f, cs = 1.0f;
        if (!dj) sincosf(sv, &sn, &cs);
        const float dads = dj ? G0[u] : fmaf(cs, G0[u + 1], -sn * G0[u]);
        const float r = dads - MFB[o];
        part += (double)r * r;
        const float v = scale * r;
        GB0[u] = dj ? v : -sn * v;
        GB0[u + 1] = dj ? 0.0f : cs * v;
    }
    red[threadIdx.x] = part;
    __syncthreads();
    for (int w = LT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) lpart[(long long)m * gridDim.x + blockIdx.x] = red[0];
}

// Column sums over the batch rows of [M][B][H] activations into the packed
// gradient: grid (ceil(H / 128), M, nvec + 1).  The last z slice adds the
// loss chunks of each member in order: loss[m] = sum lpart[m][.] / (B C).
struct ColSums {
    const float* src[RID_MAX_LAYERS + 1];
    long long dst_off[RID_MAX_LAYERS + 1];
    int n;
    const double* lpart;
    int nchunk;
    double nBC;
    float* loss;
};
__global__ void k_tr_colsum(ColSums cs, int B, int H, long long act_sm, float* __restrict__ grad, long long P) {
    pdl_trigger();
    pdl_wait();
    const int m = blockIdx.y, v = blockIdx.z;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (v == cs.n) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            double t = 0.0;
            for (int c = 0; c < cs.nchunk; ++c) t += cs.lpart[(long long)m * cs.nchunk + c];
            cs.loss[m] = (float)(t / cs.nBC);
        }
        return;
    }
    if (v > cs.n || j >= H) return;
    const float* src = cs.src[v] + (long long)m * act_sm + j;
    // rows in increasing order; eight loads are issued ahead of their adds
    float a = 0.0f;
    int b = 0;
    for (; b + 8 <= B; b += 8) {
        float x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = src[(long long)(b + k) * H];
#pragma unroll
        for (int k = 0; k < 8; ++k) a += x[k];
    }
    for (; b < B; ++b) a += src[(long long)b * H];
    grad[(long long)m * P + cs.dst_off[v] + j] = a;
}

__global__ void k_tr_adam(float* __restrict__ w, float* __restrict__ am, float* __restrict__ av,
                          const float* __restrict__ g, long long n, float lr, float b1, float b2, float eps, float c1,
                          float c2) {
    pdl_trigger();
    pdl_wait();
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float gv = g[e];
        const float m = fmaf(b1, am[e], (1.0f - b1) * gv);
        const float v = fmaf(b2, av[e], (1.0f - b2) * gv * gv);
        am[e] = m;
        av[e] = v;
        w[e] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
struct rid_trainer {
    rid_train_desc d{};
    int D = 0, P = 0;
    long long woff[RID_MAX_LAYERS] = {}, boff[RID_MAX_LAYERS] = {}, ooff = 0;
    int64_t steps = 0;
    int n_data = 0, cap_data = 0;
    float* w = nullptr;      // [M][P] parameters, then Adam m, v and the gradient
    float* am = nullptr;
    float* av = nullptr;
    float* grad = nullptr;
    float* ds = nullptr;     // data s [n][C], mf [n][C]
    float* dmf = nullptr;
    float* act = nullptr;    // activations (see carve)
    int* didx = nullptr;     // [cap_idx] batch indices
    long long cap_idx = 0;
    float* dloss = nullptr;  // [cap_loss]
    long long cap_loss = 0;
    int* dbad = nullptr;
    int* ddist = nullptr;     // [C] 1 for a distance CV, or NULL (all torsions)
    double* lpart = nullptr;  // [M][ceil(B C / 256)] loss chunk sums
    // carve of act, all [M][B][X]
    float *U, *SB, *MFB, *G0, *GB0;
    float* Q[RID_MAX_LAYERS] = {};   // dropout scales [M][B][H] per layer (NULL: no dropout)
    uint32_t dthr = 0;               // keep iff the Philox word >= dthr
    float dscale = 1.0f;             // 1 / (1 - rate)
    float *T[RID_MAX_LAYERS], *Hh[RID_MAX_LAYERS], *G[RID_MAX_LAYERS], *Dl[RID_MAX_LAYERS], *GB[RID_MAX_LAYERS],
        *TB[RID_MAX_LAYERS], *ZB[RID_MAX_LAYERS], *HB[RID_MAX_LAYERS];
};

namespace {

int tr_fail_cuda(cudaError_t e, const char* what) {
    return rid_fail(RID_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}
#define TCK(x)                                          \
    do {                                                \
        cudaError_t e_ = (x);                           \
        if (e_ != cudaSuccess) return tr_fail_cuda(e_, #x); \
    } while (0)

int grow(void** p, long long* cap, long long need, size_t elem) {
    if (need <= *cap) return RID_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc(p, (size_t)need * elem) != cudaSuccess) {
        cudaGetLastError();
        return rid_fail(RID_ERR_OOM, "trainer: cudaMalloc of %lld bytes failed", need * (long long)elem);
    }
    *cap = need;
    return RID_OK;
}

// One step's gradient into tr->grad and the per-member loss into loss[M],
// for the batch indices idx [M][B] (device) at training step `step` (the
// step index of the dropout masks).  Every kernel after the first is a
// programmatic dependent of its predecessor (pdl_wait before any access);
// the first is one too unless `after_copy` (it then follows a memory copy).
int tr_gradient(rid_trainer* tr, const int* idx, float* loss, int64_t step, bool after_copy, cudaStream_t st) {
    const rid_train_desc& d = tr->d;
    const int M = d.n_models, B = d.batch_size, C = d.n_cv, D = tr->D, L = d.n_layers, H = d.width;
    const long long P = tr->P;
    const long long smH = (long long)B * H, smD = (long long)B * D;
    {
        MaskArgs mk{tr->Q[0], L, H, (uint32_t)step, tr->dthr, (uint32_t)d.dropout_seed,
                    (uint32_t)(d.dropout_seed >> 32), tr->dscale};
        long long tot = (long long)M * B * C;
        if (mk.Q && (long long)L * M * B * ((H + 3) / 4) > tot) tot = (long long)L * M * B * ((H + 3) / 4);
        const int blocks = (int)((tot + 255) / 256 < 1024 ? (tot + 255) / 256 : 1024);
        TCK(launch_k(k_tr_gather, dim3(blocks), dim3(256), 0, st, !after_copy, idx, (const float*)tr->ds,
                     (const float*)tr->dmf, tr->n_data, M, B, C, tr->U, tr->SB, tr->MFB, tr->dbad, mk,
                     (const int*)tr->ddist));
    }
    // forward
    for (int l = 0; l < L; ++l) {
        const int fin = l == 0 ? D : H;
        GemmArgs g{};
        g.nseg = 1;
        g.seg[0].a = act_rowmajor(l == 0 ? tr->U : tr->Hh[l - 1], fin, l == 0 ? smD : smH);
        g.seg[0].b = Operand{tr->w + tr->woff[l], (long long)fin, 1, P};   // (k, j) -> W_l[j][k]
        g.seg[0].K = fin;
        g.rows = B;
        g.cols = H;
        EpiArgs& e = g.e;
        e.ld = H;
        e.act_sm = smH;
        e.bias = tr->w + tr->boff[l];
        e.bias_sm = P;
        e.T = tr->T[l];
        e.Hout = tr->Hh[l];
        e.Hin = l == 0 ? nullptr : tr->Hh[l - 1];
        e.resid = d.resnet && l >= 1;
        e.last = l == L - 1;
        e.wout = tr->w + tr->ooff;
        e.w_sm = P;
        e.Gout = tr->G[L - 1];
        e.Dout = tr->Dl[L - 1];
        e.Q = tr->Q[l];
        launch_gemm<EPI_FWD>(g, M, st, true);
    }
    // input gradient, decreasing l: g_{l-1} = d_l W_l (+ r g_l)
    for (int l = L - 1; l >= 0; --l) {
        const int fin = l == 0 ? D : H;
        GemmArgs g{};
        g.nseg = 1;
        g.seg[0].a = act_rowmajor(tr->Dl[l], H, smH);
        g.seg[0].b = Operand{tr->w + tr->woff[l], 1, (long long)fin, P};   // (k, j) -> W_l[k][j]
        g.seg[0].K = H;
        g.rows = B;
        g.cols = fin;
        EpiArgs& e = g.e;
        e.ld = fin;
        e.act_sm = l == 0 ? smD : smH;
        e.out = l == 0 ? tr->G0 : tr->G[l - 1];
        e.resid = d.resnet && l >= 1;
        e.res = tr->G[l];
        e.Tl = l == 0 ? nullptr : tr->T[l - 1];
        e.Dout = l == 0 ? nullptr : tr->Dl[l - 1];
        e.Q = l == 0 ? nullptr : tr->Q[l - 1];
        launch_gemm<EPI_BWD>(g, M, st, true);
    }
    const int nchunk = (int)(((long long)B * C + LT - 1) / LT);
    TCK(launch_k(k_tr_loss, dim3(nchunk, M), dim3(LT), 0, st, true, (const float*)tr->G0, (const float*)tr->SB,
                 (const float*)tr->MFB, B, C, tr->GB0, tr->lpart, (const int*)tr->ddist));
    // adjoint of the input-gradient pass, increasing l
    for (int l = 0; l < L; ++l) {
        const int fin = l == 0 ? D : H;
        GemmArgs g{};
        g.nseg = 1;
        g.seg[0].a = act_rowmajor(l == 0 ? tr->GB0 : tr->GB[l - 1], fin, l == 0 ? smD : smH);
        g.seg[0].b = Operand{tr->w + tr->woff[l], (long long)fin, 1, P};   // W_l^T
        g.seg[0].K = fin;
        g.rows = B;
        g.cols = H;
        EpiArgs& e = g.e;
        e.ld = H;
        e.act_sm = smH;
        e.out = tr->GB[l];
        e.resid = d.resnet && l >= 1;
        e.res = l == 0 ? nullptr : tr->GB[l - 1];
        e.Tl = tr->T[l];
        e.Gl = tr->G[l];
        e.out2 = tr->TB[l];
        e.last = l == L - 1;
        e.out3 = tr->ZB[L - 1];
        e.Q = tr->Q[l];
        launch_gemm<EPI_ADJ>(g, M, st, true);
    }
    // back through the forward pass, decreasing l (hbar_{L-1} = 0)
    for (int l = L - 1; l >= 1; --l) {
        GemmArgs g{};
        g.nseg = 1;
        g.seg[0].a = act_rowmajor(tr->ZB[l], H, smH);
        g.seg[0].b = Operand{tr->w + tr->woff[l], 1, (long long)H, P};     // W_l
        g.seg[0].K = H;
        g.rows = B;
        g.cols = H;
        EpiArgs& e = g.e;
        e.ld = H;
        e.act_sm = smH;
        e.out = tr->HB[l - 1];
        e.resid = d.resnet && l >= 1 && l < L - 1;   // hbar_{L-1} = 0
        e.res = tr->HB[l];
        e.Tl = tr->T[l - 1];
        e.tb = tr->TB[l - 1];
        e.out3 = tr->ZB[l - 1];
        e.Q = tr->Q[l - 1];
        launch_gemm<EPI_BACK>(g, M, st, true);
    }
    // weight gradients, all layers in one launch:
    // dW_l[a][b] = sum_k d_l[k][a] gbar_{l-1}[k][b] + zbar_l[k][a] h_{l-1}[k][b]
    GemmBatch wb{};
    wb.n = L;
    wb.M = M;
    for (int l = 0; l < L; ++l) {
        const int fin = l == 0 ? D : H;
        const long long smF = l == 0 ? smD : smH;
        GemmArgs& g = wb.g[l];
        g.nseg = 2;
        g.seg[0].a = act_transposed(tr->Dl[l], H, smH);
        g.seg[0].b = Operand{l == 0 ? tr->GB0 : tr->GB[l - 1], 1, (long long)fin, smF};
        g.seg[0].K = B;
        g.seg[1].a = act_transposed(tr->ZB[l], H, smH);
        g.seg[1].b = Operand{l == 0 ? tr->U : tr->Hh[l - 1], 1, (long long)fin, smF};
        g.seg[1].K = B;
        g.rows = H;
        g.cols = fin;
        g.e.out = tr->grad + tr->woff[l];
        g.e.out_sm = P;
        g.e.ld = fin;
    }
    launch_gemm_batch<EPI_STORE>(wb, st, true);
    ColSums cs{};
    for (int l = 0; l < L; ++l) {
        cs.src[l] = tr->ZB[l];
        cs.dst_off[l] = tr->boff[l];
    }
    cs.src[L] = tr->GB[L - 1];
    cs.dst_off[L] = tr->ooff;
    cs.n = L + 1;
    cs.lpart = tr->lpart;
    cs.nchunk = nchunk;
    cs.nBC = (double)B * C;
    cs.loss = loss;
    TCK(launch_k(k_tr_colsum, dim3((H + 127) / 128, M, L + 2), dim3(128), 0, st, true, cs, B, H, smH, tr->grad,
                 (long long)P));
    return RID_OK;
}

int tr_check_desc(const rid_train_desc* d) {
    if (!d) return rid_fail(RID_ERR_ARG, "trainer: desc is NULL");
    if (d->n_models < 1 || d->n_models > RID_MAX_MODELS) return rid_fail(RID_ERR_ARG, "trainer: n_models out of range");
    if (d->n_cv < 1 || d->n_cv > RID_MAX_CV) return rid_fail(RID_ERR_ARG, "trainer: n_cv out of range");
    if (d->n_layers < 1 || d->n_layers > RID_MAX_LAYERS) return rid_fail(RID_ERR_ARG, "trainer: n_layers out of range");
    if (d->width < 1 || d->width > RID_MAX_WIDTH) return rid_fail(RID_ERR_ARG, "trainer: width out of range");
    if (d->batch_size < 1 || d->batch_size > 65536) return rid_fail(RID_ERR_ARG, "trainer: batch_size out of range");
    if (!(d->init_lr > 0) || !(d->decay_rate > 0) || d->decay_steps < 1)
        return rid_fail(RID_ERR_ARG, "trainer: learning-rate schedule out of range");
    if (!(d->beta1 >= 0 && d->beta1 < 1) || !(d->beta2 >= 0 && d->beta2 < 1) || !(d->adam_eps > 0))
        return rid_fail(RID_ERR_ARG, "trainer: Adam parameters out of range");
    if (!(d->dropout_rate >= 0 && d->dropout_rate < 1)) return rid_fail(RID_ERR_ARG, "trainer: dropout_rate outside [0, 1)");
    return RID_OK;
}

int tr_copy_in(void* dst, const void* src, size_t bytes, int mem, cudaStream_t st) {
    TCK(cudaMemcpyAsync(dst, src, bytes, mem == RID_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    return RID_OK;
}
int tr_copy_out(void* dst, const void* src, size_t bytes, int mem, cudaStream_t st) {
    TCK(cudaMemcpyAsync(dst, src, bytes, mem == RID_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    return RID_OK;
}

int tr_finish(rid_trainer* tr, cudaStream_t st) {
    int bad = 0;
    TCK(cudaMemcpyAsync(&bad, tr->dbad, sizeof(int), cudaMemcpyDeviceToHost, st));
    TCK(cudaStreamSynchronize(st));
    TCK(cudaGetLastError());
    if (bad) {
        TCK(cudaMemsetAsync(tr->dbad, 0, sizeof(int), st));
        TCK(cudaStreamSynchronize(st));
        return rid_fail(RID_ERR_ARG, "trainer: a batch index is outside [0, n_data)");
    }
    return RID_OK;
}

}  // namespace

extern "C" {

RID_API int rid_trainer_create(const rid_train_desc* desc, const float* weights, rid_trainer** out) {
    if (!out || !weights) return rid_fail(RID_ERR_ARG, "trainer: NULL argument");
    *out = nullptr;
    if (int rc = tr_check_desc(desc)) return rc;
    rid_trainer* tr = new rid_trainer();
    tr->d = *desc;
    const int M = desc->n_models, C = desc->n_cv, L = desc->n_layers, H = desc->width, B = desc->batch_size;
    const int D = 2 * C;
    tr->D = D;
    long long o = 0;
    int fin = D;
    for (int l = 0; l < L; ++l) {
        tr->woff[l] = o;
        o += (long long)H * fin;
        tr->boff[l] = o;
        o += H;
        fin = H;
    }
    tr->ooff = o;
    o += H + 1;
    tr->P = (int)o;
    const long long nP = (long long)M * tr->P;
    const long long smH = (long long)B * H, smD = (long long)B * D, smC = (long long)B * C;
    // activations: U, G0, GB0 [M][B][D]; SB, MFB [M][B][C]; per layer T, Hh (resnet or dropout), G, Dl, GB,
    // TB, ZB, HB, and Q (dropout)
    const bool drop = desc->dropout_rate > 0;
    const long long per_layer = ((desc->resnet || drop ? 8 : 7) + (drop ? 1 : 0)) * smH;
    const long long nact = (long long)M * (3 * smD + 2 * smC + L * per_layer);
    bool ok = cudaMalloc(&tr->w, sizeof(float) * 4 * nP) == cudaSuccess;
    ok = ok && cudaMalloc(&tr->act, sizeof(float) * nact) == cudaSuccess;
    ok = ok && cudaMalloc(&tr->dbad, sizeof(int)) == cudaSuccess;
    ok = ok && cudaMalloc(&tr->lpart, sizeof(double) * M * (((long long)B * C + 255) / 256)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        rid_trainer_destroy(tr);
        return rid_fail(RID_ERR_OOM, "trainer: device allocation failed");
    }
    tr->am = tr->w + nP;
    tr->av = tr->am + nP;
    tr->grad = tr->av + nP;
    float* p = tr->act;
    auto take = [&](long long per_member) { float* r = p; p += M * per_member; return r; };
    tr->U = take(smD);
    tr->G0 = take(smD);
    tr->GB0 = take(smD);
    tr->SB = take(smC);
    tr->MFB = take(smC);
    for (int l = 0; l < L; ++l) {
        tr->T[l] = take(smH);
        tr->Hh[l] = desc->resnet || drop ? take(smH) : tr->T[l];
        tr->G[l] = take(smH);
        tr->Dl[l] = take(smH);
        tr->GB[l] = take(smH);
        tr->TB[l] = take(smH);
        tr->ZB[l] = take(smH);
        tr->HB[l] = take(smH);
    }
    if (drop) {   // the scales of all layers are contiguous: k_tr_mask writes them in one launch
        for (int l = 0; l < L; ++l) tr->Q[l] = take(smH);
        tr->dthr = (uint32_t)std::floor(desc->dropout_rate * 4294967296.0);
        tr->dscale = (float)(1.0 / (1.0 - desc->dropout_rate));
    }
    bool any_dist = false;
    for (int j = 0; desc->cv_dist && j < C; ++j) any_dist |= desc->cv_dist[j] != 0;
    if (any_dist) {
        std::vector<int> h(C);
        for (int j = 0; j < C; ++j) h[j] = desc->cv_dist[j] ? 1 : 0;
        if (cudaMalloc(&tr->ddist, sizeof(int) * C) != cudaSuccess ||
            cudaMemcpy(tr->ddist, h.data(), sizeof(int) * C, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            rid_trainer_destroy(tr);
            return rid_fail(RID_ERR_OOM, "trainer: device allocation failed");
        }
    }
    tr->d.cv_dist = nullptr;   // the caller's array is not kept
    if (cudaMemcpy(tr->w, weights, sizeof(float) * nP, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(tr->am, 0, sizeof(float) * 3 * nP) != cudaSuccess || cudaMemset(tr->act, 0, sizeof(float) * nact) != cudaSuccess ||
        cudaMemset(tr->dbad, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        rid_trainer_destroy(tr);
        return rid_fail(RID_ERR_CUDA, "trainer: initial copy failed");
    }
    *out = tr;
    return RID_OK;
}

RID_API int rid_trainer_destroy(rid_trainer* tr) {
    if (!tr) return RID_OK;
    cudaFree(tr->w);
    cudaFree(tr->act);
    cudaFree(tr->dbad);
    cudaFree(tr->ddist);
    cudaFree(tr->lpart);
    cudaFree(tr->ds);
    cudaFree(tr->didx);
    cudaFree(tr->dloss);
    delete tr;
    return RID_OK;
}

RID_API int rid_trainer_set_data(rid_trainer* tr, int32_t n, const float* s, const float* mf, int32_t mem, void* stream) {
    if (!tr || !s || !mf || n < 1) return rid_fail(RID_ERR_ARG, "trainer: bad data arguments");
    if (mem != RID_MEM_HOST && mem != RID_MEM_DEVICE) return rid_fail(RID_ERR_ARG, "trainer: bad mem");
    cudaStream_t st = (cudaStream_t)stream;
    const int C = tr->d.n_cv;
    if (n > tr->cap_data) {
        cudaFree(tr->ds);
        tr->ds = nullptr;
        tr->cap_data = 0;
        if (cudaMalloc(&tr->ds, sizeof(float) * 2 * (size_t)n * C) != cudaSuccess) {
            cudaGetLastError();
            return rid_fail(RID_ERR_OOM, "trainer: data allocation failed");
        }
        tr->cap_data = n;
    }
    tr->dmf = tr->ds + (size_t)tr->cap_data * C;
    tr->n_data = n;
    if (int rc = tr_copy_in(tr->ds, s, sizeof(float) * (size_t)n * C, mem, st)) return rc;
    if (int rc = tr_copy_in(tr->dmf, mf, sizeof(float) * (size_t)n * C, mem, st)) return rc;
    TCK(cudaStreamSynchronize(st));
    return RID_OK;
}

RID_API int rid_trainer_grad(rid_trainer* tr, const int32_t* idx, float* loss_out, float* grad_out, int32_t mem,
                             void* stream) {
    NvtxScope nvtx_("rid_trainer_grad");
    if (!tr || !idx) return rid_fail(RID_ERR_ARG, "trainer: NULL argument");
    if (mem != RID_MEM_HOST && mem != RID_MEM_DEVICE) return rid_fail(RID_ERR_ARG, "trainer: bad mem");
    if (tr->n_data < 1) return rid_fail(RID_ERR_STATE, "trainer: no data set");
    cudaStream_t st = (cudaStream_t)stream;
    const int M = tr->d.n_models, B = tr->d.batch_size;
    if (int rc = grow((void**)&tr->didx, &tr->cap_idx, (long long)M * B, sizeof(int))) return rc;
    if (int rc = grow((void**)&tr->dloss, &tr->cap_loss, M, sizeof(float))) return rc;
    if (int rc = tr_copy_in(tr->didx, idx, sizeof(int) * (size_t)M * B, mem, st)) return rc;
    if (int rc = tr_gradient(tr, tr->didx, tr->dloss, tr->steps, true, st)) return rc;
    TCK(cudaGetLastError());
    if (loss_out)
        if (int rc = tr_copy_out(loss_out, tr->dloss, sizeof(float) * M, mem, st)) return rc;
    if (grad_out)
        if (int rc = tr_copy_out(grad_out, tr->grad, sizeof(float) * (size_t)M * tr->P, mem, st)) return rc;
    return tr_finish(tr, st);
}

RID_API int rid_trainer_run(rid_trainer* tr, int32_t n_steps, const int32_t* idx, float* loss_out, int32_t mem,
                            void* stream) {
    NvtxScope nvtx_("rid_trainer_run");
    if (!tr || !idx || n_steps < 0) return rid_fail(RID_ERR_ARG, "trainer: bad run arguments");
    if (mem != RID_MEM_HOST && mem != RID_MEM_DEVICE) return rid_fail(RID_ERR_ARG, "trainer: bad mem");
    if (tr->n_data < 1) return rid_fail(RID_ERR_STATE, "trainer: no data set");
    if (n_steps == 0) return RID_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const rid_train_desc& d = tr->d;
    const int M = d.n_models, B = d.batch_size;
    const long long per = (long long)M * B;
    if (int rc = grow((void**)&tr->didx, &tr->cap_idx, per * n_steps, sizeof(int))) return rc;
    if (int rc = grow((void**)&tr->dloss, &tr->cap_loss, (long long)M * n_steps, sizeof(float))) return rc;
    if (int rc = tr_copy_in(tr->didx, idx, sizeof(int) * (size_t)(per * n_steps), mem, st)) return rc;
    const long long nP = (long long)M * tr->P;
    const int ablocks = (int)((nP + 255) / 256 < 2048 ? (nP + 255) / 256 : 2048);
    for (int k = 0; k < n_steps; ++k) {
        const int64_t t = tr->steps + k;
        if (int rc = tr_gradient(tr, tr->didx + per * k, tr->dloss + (long long)M * k, t, k == 0, st)) return rc;
        const double lr = d.init_lr * std::pow(d.decay_rate, (double)t / (double)d.decay_steps);
        const double c1 = 1.0 - std::pow(d.beta1, (double)(t + 1)), c2 = 1.0 - std::pow(d.beta2, (double)(t + 1));
        TCK(launch_k(k_tr_adam, dim3(ablocks), dim3(256), 0, st, true, tr->w, tr->am, tr->av, (const float*)tr->grad,
                     nP, (float)lr, (float)d.beta1, (float)d.beta2, (float)d.adam_eps, (float)c1, (float)c2));
    }
    TCK(cudaGetLastError());
    if (loss_out)
        if (int rc = tr_copy_out(loss_out, tr->dloss, sizeof(float) * (size_t)M * n_steps, mem, st)) return rc;
    const int rc = tr_finish(tr, st);
    if (rc == RID_OK) tr->steps += n_steps;
    return rc;
}

RID_API int rid_trainer_weights(rid_trainer* tr, float* weights_out, int64_t* steps_done, int32_t mem, void* stream) {
    if (!tr) return rid_fail(RID_ERR_ARG, "trainer: NULL argument");
    if (mem != RID_MEM_HOST && mem != RID_MEM_DEVICE) return rid_fail(RID_ERR_ARG, "trainer: bad mem");
    cudaStream_t st = (cudaStream_t)stream;
    if (weights_out)
        if (int rc = tr_copy_out(weights_out, tr->w, sizeof(float) * (size_t)tr->d.n_models * tr->P, mem, st)) return rc;
    if (steps_done) *steps_done = tr->steps;
    TCK(cudaStreamSynchronize(st));
    return RID_OK;
}

}  // extern "C"
