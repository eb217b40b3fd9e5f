// k_mcmc.cu -- MCMC dimension reduction of the trained ensemble (Sec.
// "Dimension reduction phase": numb_walkers, numb_steps, temperature, bins,
// proj_cv_index; Introduction, automatic PMF calculation).
//
// W walkers run Metropolis Monte Carlo in CV space on the ensemble-mean free
// energy Abar(s) = (1/M) sum_i A_i(s) at temperature kT.  Every step:
//   k_mc_propose  s' = wrap(s + step_size xi) (a distance CV: not wrapped),
//                 xi: normal c % 3 of the Box-Muller triple of Philox counter
//                 (c / 3, walker, step, 2); writes the MLP input
//                 u' = (cos s', sin s') (a distance CV: (s', 0))
//   forward GEMMs one batched FP32 GEMM per layer (rid_gemm.cuh), members on
//                 grid z, the input u' shared by all members
//   k_mc_accept   one warp per walker: A_i = w_out . h + b_out, Abar' as the
//                 mean in member order; accept iff kT ln u + (Abar' - Abar) < 0
//                 and every distance CV of s' lies in its range [lo, hi]
//                 with u = (x + 1/2) 2^-32, x = word 0 of counter
//                 (0, walker, step, 3); from step n_burn on, the current state
//                 of every walker is counted into one histogram per CV and one
//                 2-D histogram of a CV pair (integer atomics: exact)
// and at the end k_mc_pmf turns the counts into -kT ln(count / total),
// shifted to a zero minimum (+inf for empty bins).  With path nodes, the warp
// also maps each counted state onto the path collective variables (lanes over
// the nodes, the smallest distance factored out, sums in a fixed order) and
// counts (s_path, z_path).
#include <cmath>
#include <vector>

#include "rid_gemm.cuh"

namespace {

constexpr float MC_PI = 3.14159265358979f;
constexpr float MC_INV_2PI = 0.159154943091895f;

// bin of an angle in [-pi, pi): floor((v + pi) / (2 pi) * bins), each
// operation rounded once, clamped to [0, bins - 1]
__device__ __forceinline__ int mc_bin(float v, int bins) {
    const float t = __fmul_rn(__fmul_rn(__fadd_rn(v, MC_PI), MC_INV_2PI), (float)bins);
    int b = (int)floorf(t);
    return b < 0 ? 0 : (b >= bins ? bins - 1 : b);
}
// bin of CV c: the angle bin for a torsion, floor((v - lo) / (hi - lo) * bins)
// (each operation rounded once) for a distance CV, clamped
__device__ __forceinline__ int mc_bin_cv(float v, int c, int bins, const McCvDev& k) {
    if (!(k.dist && k.dist[c])) return mc_bin(v, bins);
    const float t = __fmul_rn(__fdiv_rn(__fsub_rn(v, k.lo[c]), __fsub_rn(k.hi[c], k.lo[c])), (float)bins);
    int b = (int)floorf(t);
    return b < 0 ? 0 : (b >= bins ? bins - 1 : b);
}
// MLP input pair of CV c: (cos v, sin v) for a torsion, (v, 0) for a distance
__device__ __forceinline__ void mc_input(float v, bool dist, float* U) {
    if (dist) {
        U[0] = v;
        U[1] = 0.0f;
    } else {
        float sn, cs;
        sincosf(v, &sn, &cs);
        U[0] = cs;
        U[1] = sn;
    }
}

__global__ void k_mc_features(const float* __restrict__ s, float* __restrict__ U, long long n, int C, McCvDev k) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        mc_input(s[e], k.dist && k.dist[(int)(e % C)], U + 2 * e);
}

__global__ void k_mc_propose(const float* __restrict__ s, float* __restrict__ sp, float* __restrict__ U, int W, int C,
                             uint32_t step, float step_size, uint32_t k0, uint32_t k1, McCvDev k) {
    const long long n = (long long)W * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int w = (int)(e / C), c = (int)(e - (long long)w * C);
        const float3 z = rid_normals3(rid_philox(make_uint4((uint32_t)(c / 3), (uint32_t)w, step, 2u), k0, k1));
        const int r = c % 3;
        const float xi = r == 0 ? z.x : (r == 1 ? z.y : z.z);
        const bool dist = k.dist && k.dist[c];
        const float v = dist ? fmaf(step_size, xi, s[e]) : rid_wrapf(fmaf(step_size, xi, s[e]));
        sp[e] = v;
        mc_input(v, dist, U + 2 * e);
    }
}

struct AcceptArgs {
    const float* h;        // [M][W][H] last hidden layer
    const float* w;        // [M][P] packed weights
    long long P, ooff;     // floats per member, offset of w_out (b_out follows)
    int M, W, H, C;
    float* s;              // [W][C] state
    const float* sp;       // [W][C] proposal
    float* A;              // [W] Abar at the state
    uint32_t step, k0, k1;
    float kT;
    int init;              // 1: A = Abar(s) only
    int count;             // count the states into the histograms
    int bins, pi, pj;
    unsigned long long* hist1;   // [C][bins]
    unsigned long long* hist2;   // [bins][bins]
    unsigned long long* nacc;
    // path projection (npath = 0: off)
    int npath, Cp;
    const int* pcv;              // [Cp]
    const float* pnodes;         // [P][Cp]
    float lam, z_lo, z_hi;
    unsigned long long* histp;   // [bins][bins]
    // member values from a system's ensemble kernels ([na][W], na = M x slices) instead of h . w_out
    const float* aval;
    int na;
    McCvDev cvk;                 // distance CVs: range, bins, plain path differences
};

__global__ void k_mc_accept(AcceptArgs a) {
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= a.W) return;                       // whole warps only
    float abar = 0.0f;
    if (a.aval) {
        float part = 0.0f;
        for (int k = lane; k < a.na; k += 32) part += a.aval[(long long)k * a.W + w];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        abar = part;
    } else {
        for (int m = 0; m < a.M; ++m) {
            const float* wo = a.w + (long long)m * a.P + a.ooff;
            const float* h = a.h + ((long long)m * a.W + w) * a.H;
            float part = 0.0f;
            for (int j = lane; j < a.H; j += 32) part = fmaf(wo[j], h[j], part);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            abar += part + wo[a.H];
        }
    }
    abar /= (float)a.M;
    float* s = a.s + (long long)w * a.C;
    if (a.init) {
        if (lane == 0) a.A[w] = abar;
        return;
    }
    const uint4 r = rid_philox(make_uint4(0u, (uint32_t)w, a.step, 3u), a.k0, a.k1);
    const float margin = (abar - a.A[w]) - 0.5f * a.kT * rid_m2logu(r.x);   // kT ln u + dAbar
    // a proposal that takes a distance CV out of its range is refused
    bool inside = true;
    if (a.cvk.dist) {
        const float* sp = a.sp + (long long)w * a.C;
        for (int c = lane; c < a.C; c += 32)
            if (a.cvk.dist[c] && !(sp[c] >= a.cvk.lo[c] && sp[c] <= a.cvk.hi[c])) inside = false;
        inside = __all_sync(0xffffffffu, inside);
    }
    if (margin < 0.0f && inside) {
        const float* sp = a.sp + (long long)w * a.C;
        for (int c = lane; c < a.C; c += 32) s[c] = sp[c];
        if (lane == 0) {
            a.A[w] = abar;
            atomicAdd(a.nacc, 1ull);
        }
    }
    __syncwarp();
    if (a.count) {
        for (int c = lane; c < a.C; c += 32)
            atomicAdd(&a.hist1[(long long)c * a.bins + mc_bin_cv(s[c], c, a.bins, a.cvk)], 1ull);
        if (lane == 0 && a.hist2)
            atomicAdd(&a.hist2[(long long)mc_bin_cv(s[a.pi], a.pi, a.bins, a.cvk) * a.bins +
                               mc_bin_cv(s[a.pj], a.pj, a.bins, a.cvk)],
                      1ull);
        if (a.npath > 0) {
            // d_i for the nodes of this lane, then the smallest over the warp
            float dmin = INFINITY;
            for (int i = lane; i < a.npath; i += 32) {
                float d2 = 0.0f;
                for (int c = 0; c < a.Cp; ++c) {
                    const int cv = a.pcv[c];
                    const float dd = s[cv] - a.pnodes[(long long)i * a.Cp + c];
                    const float d = (a.cvk.dist && a.cvk.dist[cv]) ? dd : rid_wrapf(dd);
                    d2 = fmaf(d, d, d2);
                }
                dmin = fminf(dmin, d2);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
            float s0 = 0.0f, s1 = 0.0f;
            for (int i = lane; i < a.npath; i += 32) {
                float d2 = 0.0f;
                for (int c = 0; c < a.Cp; ++c) {
                    const int cv = a.pcv[c];
                    const float dd = s[cv] - a.pnodes[(long long)i * a.Cp + c];
                    const float d = (a.cvk.dist && a.cvk.dist[cv]) ? dd : rid_wrapf(dd);
                    d2 = fmaf(d, d, d2);
                }
                const float e = expf(-a.lam * (d2 - dmin));
                s0 += e;
                s1 = fmaf((float)(i + 1), e, s1);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            }
            if (lane == 0) {
                const float sp = s1 / s0, z = dmin - logf(s0) / a.lam;
                int bs = (int)floorf((sp - 1.0f) / (float)(a.npath - 1) * (float)a.bins);
                int bz = (int)floorf((z - a.z_lo) / (a.z_hi - a.z_lo) * (float)a.bins);
                bs = bs < 0 ? 0 : (bs >= a.bins ? a.bins - 1 : bs);
                bz = bz < 0 ? 0 : (bz >= a.bins ? a.bins - 1 : bz);
                atomicAdd(&a.histp[(long long)bs * a.bins + bz], 1ull);
            }
        }
    }
}

// One CTA per histogram row of length n: f = -kT ln(count / total) - min f.
constexpr int PT = 256;
__global__ void __launch_bounds__(PT) k_mc_pmf(const unsigned long long* __restrict__ hist, int n, double kT,
                                               double* __restrict__ pmf) {
    __shared__ unsigned long long tot_s[PT];
    __shared__ double min_s[PT];
    const unsigned long long* h = hist + (long long)blockIdx.x * n;
    double* f = pmf + (long long)blockIdx.x * n;
    unsigned long long tot = 0;
    for (int i = threadIdx.x; i < n; i += PT) tot += h[i];
    tot_s[threadIdx.x] = tot;
    __syncthreads();
    for (int k = PT / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) tot_s[threadIdx.x] += tot_s[threadIdx.x + k];
        __syncthreads();
    }
    const double total = (double)tot_s[0];
    double mn = INFINITY;
    for (int i = threadIdx.x; i < n; i += PT)
        if (h[i]) mn = fmin(mn, -kT * log((double)h[i] / total));
    min_s[threadIdx.x] = mn;
    __syncthreads();
    for (int k = PT / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) min_s[threadIdx.x] = fmin(min_s[threadIdx.x], min_s[threadIdx.x + k]);
        __syncthreads();
    }
    mn = min_s[0];
    for (int i = threadIdx.x; i < n; i += PT) f[i] = h[i] ? -kT * log((double)h[i] / total) - mn : INFINITY;
}

int mc_cuda(cudaError_t e, const char* what) { return rid_fail(RID_ERR_CUDA, "mcmc: %s: %s", what, cudaGetErrorString(e)); }

struct McBufs {
    void* p = nullptr;
    ~McBufs() {
        if (p) cudaFree(p);
    }
};

}  // namespace

int rid_mc_range_check(int C, const int32_t* dist, const double* lo, const double* hi) {
    if (!dist) return RID_OK;
    if (!lo || !hi) return rid_fail(RID_ERR_ARG, "mcmc: distance CVs need cv_lo and cv_hi");
    for (int c = 0; c < C; ++c)
        if (dist[c] && !(std::isfinite(lo[c]) && std::isfinite(hi[c]) && lo[c] < hi[c]))
            return rid_fail(RID_ERR_ARG, "mcmc: distance CV %d needs finite cv_lo < cv_hi", c);
    return RID_OK;
}

int rid_mc_path_check(int NP, int Cp, int C, const int32_t* cv, const float* nodes, double lambda, double z_lo,
                      double z_hi) {
    if (NP == 0) return RID_OK;
    if (NP < 2 || NP > 1024 || Cp < 1 || Cp > C || !cv || !nodes || !(lambda > 0) || !(z_hi > z_lo))
        return rid_fail(RID_ERR_ARG, "mcmc: path projection parameters out of range");
    for (int c = 0; c < Cp; ++c)
        if (cv[c] < 0 || cv[c] >= C) return rid_fail(RID_ERR_ARG, "mcmc: path CV index out of range");
    return RID_OK;
}

extern "C" RID_API int rid_mcmc(const rid_mcmc_desc* d, const float* s0, float* s_out, uint64_t* hist1_out,
                                uint64_t* hist2_out, double* pmf1_out, double* pmf2_out, uint64_t* histp_out,
                                double* pmfp_out, int64_t* n_accepted, int32_t mem, void* stream) {
    NvtxScope nvtx_("rid_mcmc");
    if (!d || !s0 || !d->weights) return rid_fail(RID_ERR_ARG, "mcmc: NULL argument");
    if (mem != RID_MEM_HOST && mem != RID_MEM_DEVICE) return rid_fail(RID_ERR_ARG, "mcmc: bad mem");
    const int M = d->n_models, C = d->n_cv, L = d->n_layers, H = d->width, W = d->n_walkers, bins = d->bins;
    if (M < 1 || M > RID_MAX_MODELS || C < 1 || C > RID_MAX_CV || L < 1 || L > RID_MAX_LAYERS || H < 1 ||
        H > RID_MAX_WIDTH || W < 1 || W > (1 << 24))
        return rid_fail(RID_ERR_ARG, "mcmc: ensemble or walker count out of range");
    if (d->n_steps < 0 || d->n_steps > 0xFFFFFFFFll || d->n_burn < 0 || !(d->kT > 0) || !(d->step_size >= 0) ||
        bins < 1 || bins > 4096 || d->proj_i < 0 || d->proj_i >= C || d->proj_j < 0 || d->proj_j >= C)
        return rid_fail(RID_ERR_ARG, "mcmc: run parameters out of range");
    const int NP = d->path_n_nodes, Cp = d->path_n_cv;
    if (int r = rid_mc_path_check(NP, Cp, C, d->path_cv, d->path_nodes, d->path_lambda, d->path_z_lo, d->path_z_hi))
        return r;
    if (int r = rid_mc_range_check(C, d->cv_dist, d->cv_lo, d->cv_hi)) return r;
    const bool has_dist = d->cv_dist != nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    const int D = 2 * C;
    long long woff[RID_MAX_LAYERS], boff[RID_MAX_LAYERS], o = 0;
    for (int l = 0, fin = D; l < L; ++l, fin = H) {
        woff[l] = o;
        o += (long long)H * fin;
        boff[l] = o;
        o += H;
    }
    const long long ooff = o, P = o + H + 1;
    // device memory, carved from one allocation (released on return)
    const long long nW = (long long)M * P, nS = (long long)W * C, nU = (long long)W * D, nH = (long long)M * W * H;
    const long long n1 = (long long)C * bins, n2 = (long long)bins * bins;
    const size_t bytes_f = sizeof(float) * (size_t)(nW + 2 * nS + W + nU + (d->resnet ? 3 : 2) * nH);
    const long long np2 = NP ? n2 : 0, npn = (long long)NP * Cp;
    const size_t bytes_u = sizeof(unsigned long long) * (size_t)(n1 + n2 + np2 + 1);
    const size_t bytes_d = sizeof(double) * (size_t)(n1 + n2 + np2);
    const size_t bytes_p = sizeof(float) * (size_t)npn + sizeof(int) * (size_t)Cp;
    const size_t bytes_k = has_dist ? (sizeof(int) + 2 * sizeof(float)) * (size_t)C : 0;
    McBufs buf;
    if (cudaMalloc(&buf.p, bytes_u + bytes_d + bytes_f + bytes_p + bytes_k) != cudaSuccess) {
        cudaGetLastError();
        return rid_fail(RID_ERR_OOM, "mcmc: device allocation of %zu bytes failed",
                        bytes_u + bytes_d + bytes_f + bytes_p + bytes_k);
    }
    unsigned long long* hist1 = reinterpret_cast<unsigned long long*>(buf.p);
    unsigned long long* hist2 = hist1 + n1;
    unsigned long long* histp = hist2 + n2;
    unsigned long long* nacc = histp + np2;
    double* pmf1 = reinterpret_cast<double*>(nacc + 1);
    double* pmf2 = pmf1 + n1;
    double* pmfp = pmf2 + n2;
    float* wts = reinterpret_cast<float*>(pmfp + np2);
    float* s = wts + nW;
    float* sp = s + nS;
    float* A = sp + nS;
    float* U = A + W;
    float* hb[2] = {U + nU, U + nU + nH};
    float* tb = d->resnet ? hb[1] + nH : nullptr;
    float* pnodes = (d->resnet ? tb + nH : hb[1] + nH);
    int* pcv = reinterpret_cast<int*>(pnodes + npn);
    McCvDev cvk;
    if (has_dist) {
        int* kd = pcv + Cp;
        float* klo = reinterpret_cast<float*>(kd + C);
        std::vector<int> hd(C);
        std::vector<float> hr(2 * (size_t)C, 0.0f);
        for (int c = 0; c < C; ++c) {
            hd[c] = d->cv_dist[c] ? 1 : 0;
            if (hd[c]) {
                hr[c] = (float)d->cv_lo[c];
                hr[C + c] = (float)d->cv_hi[c];
            }
        }
        cudaError_t e1 = cudaMemcpyAsync(kd, hd.data(), sizeof(int) * C, cudaMemcpyHostToDevice, (cudaStream_t)stream);
        if (e1 == cudaSuccess)
            e1 = cudaMemcpyAsync(klo, hr.data(), sizeof(float) * 2 * C, cudaMemcpyHostToDevice, (cudaStream_t)stream);
        if (e1 == cudaSuccess) e1 = cudaStreamSynchronize((cudaStream_t)stream);   // host staging goes out of scope
        if (e1 != cudaSuccess) return mc_cuda(e1, "CV ranges");
        cvk.dist = kd;
        cvk.lo = klo;
        cvk.hi = klo + C;
    }
    const cudaMemcpyKind kin = mem == RID_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind kout = mem == RID_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(wts, d->weights, sizeof(float) * nW, kin, st)) != cudaSuccess) return mc_cuda(e, "weights");
    if ((e = cudaMemcpyAsync(s, s0, sizeof(float) * nS, kin, st)) != cudaSuccess) return mc_cuda(e, "s0");
    if ((e = cudaMemsetAsync(hist1, 0, bytes_u, st)) != cudaSuccess) return mc_cuda(e, "memset");
    if (NP) {
        if ((e = cudaMemcpyAsync(pnodes, d->path_nodes, sizeof(float) * npn, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return mc_cuda(e, "path nodes");
        if ((e = cudaMemcpyAsync(pcv, d->path_cv, sizeof(int) * Cp, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return mc_cuda(e, "path CVs");
    }

    const uint32_t k0 = (uint32_t)d->seed, k1 = (uint32_t)(d->seed >> 32);
    const int eb = (int)((nS + 255) / 256 < 4096 ? (nS + 255) / 256 : 4096);
    auto forward = [&]() {
        for (int l = 0; l < L; ++l) {
            const int fin = l == 0 ? D : H;
            GemmArgs g{};
            g.nseg = 1;
            g.seg[0].a = l == 0 ? act_rowmajor(U, D, 0) : act_rowmajor(hb[(l - 1) & 1], H, (long long)W * H);
            g.seg[0].b = Operand{wts + woff[l], (long long)fin, 1, P};      // (k, j) -> W_l[j][k]
            g.seg[0].K = fin;
            g.rows = W;
            g.cols = H;
            EpiArgs& ea = g.e;
            ea.ld = H;
            ea.act_sm = (long long)W * H;
            ea.bias = wts + boff[l];
            ea.bias_sm = P;
            ea.Hout = hb[l & 1];
            ea.T = d->resnet ? tb : ea.Hout;
            ea.Hin = l == 0 ? nullptr : hb[(l - 1) & 1];
            ea.resid = d->resnet && l >= 1;
            launch_gemm<EPI_FWD>(g, M, st);
        }
    };
    AcceptArgs aa{};
    aa.h = hb[(L - 1) & 1];
    aa.w = wts;
    aa.P = P;
    aa.ooff = ooff;
    aa.M = M;
    aa.W = W;
    aa.H = H;
    aa.C = C;
    aa.s = s;
    aa.sp = sp;
    aa.A = A;
    aa.k0 = k0;
    aa.k1 = k1;
    aa.kT = (float)d->kT;
    aa.bins = bins;
    aa.pi = d->proj_i;
    aa.pj = d->proj_j;
    aa.hist1 = hist1;
    aa.hist2 = hist2;
    aa.nacc = nacc;
    aa.npath = NP;
    aa.Cp = Cp;
    aa.pcv = pcv;
    aa.pnodes = pnodes;
    aa.lam = (float)d->path_lambda;
    aa.z_lo = (float)d->path_z_lo;
    aa.z_hi = (float)d->path_z_hi;
    aa.histp = histp;
    aa.cvk = cvk;
    const int wpb = 4;                                  // walkers (warps) per CTA
    const int ab = (W + wpb - 1) / wpb;
    k_mc_features<<<eb, 256, 0, st>>>(s, U, nS, C, cvk);
    forward();
    aa.init = 1;
    k_mc_accept<<<ab, 32 * wpb, 0, st>>>(aa);
    aa.init = 0;
    for (int64_t t = 0; t < d->n_steps; ++t) {
        k_mc_propose<<<eb, 256, 0, st>>>(s, sp, U, W, C, (uint32_t)t, (float)d->step_size, k0, k1, cvk);
        forward();
        aa.step = (uint32_t)t;
        aa.count = t >= d->n_burn;
        k_mc_accept<<<ab, 32 * wpb, 0, st>>>(aa);
    }
    k_mc_pmf<<<C, PT, 0, st>>>(hist1, bins, d->kT, pmf1);
    k_mc_pmf<<<1, PT, 0, st>>>(hist2, (int)n2, d->kT, pmf2);
    if (NP) k_mc_pmf<<<1, PT, 0, st>>>(histp, (int)n2, d->kT, pmfp);
    if ((e = cudaGetLastError()) != cudaSuccess) return mc_cuda(e, "launch");
    if (s_out && (e = cudaMemcpyAsync(s_out, s, sizeof(float) * nS, kout, st)) != cudaSuccess) return mc_cuda(e, "s_out");
    if (hist1_out && (e = cudaMemcpyAsync(hist1_out, hist1, sizeof(uint64_t) * n1, kout, st)) != cudaSuccess)
        return mc_cuda(e, "hist1");
    if (hist2_out && (e = cudaMemcpyAsync(hist2_out, hist2, sizeof(uint64_t) * n2, kout, st)) != cudaSuccess)
        return mc_cuda(e, "hist2");
    if (pmf1_out && (e = cudaMemcpyAsync(pmf1_out, pmf1, sizeof(double) * n1, kout, st)) != cudaSuccess)
        return mc_cuda(e, "pmf1");
    if (pmf2_out && (e = cudaMemcpyAsync(pmf2_out, pmf2, sizeof(double) * n2, kout, st)) != cudaSuccess)
        return mc_cuda(e, "pmf2");
    if (NP && histp_out && (e = cudaMemcpyAsync(histp_out, histp, sizeof(uint64_t) * n2, kout, st)) != cudaSuccess)
        return mc_cuda(e, "hist_path");
    if (NP && pmfp_out && (e = cudaMemcpyAsync(pmfp_out, pmfp, sizeof(double) * n2, kout, st)) != cudaSuccess)
        return mc_cuda(e, "pmf_path");
    unsigned long long na = 0;
    if ((e = cudaMemcpyAsync(&na, nacc, sizeof(na), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return mc_cuda(e, "nacc");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return mc_cuda(e, "synchronize");
    if (n_accepted) *n_accepted = (int64_t)na;
    return RID_OK;
}

// ---------------------------------------------------------------------------
// Launchers for rid_mcmc_system (rid_api.cu), which evaluates the ensemble
// with a system's own kernels and precision.
void rid_launch_mc_features(const float* s, float* U, long long n, int C, const McCvDev& cvk, cudaStream_t st) {
    const int eb = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_mc_features<<<eb, 256, 0, st>>>(s, U, n, C, cvk);
}

void rid_launch_mc_propose(const float* s, float* sp, float* U, int W, int C, uint32_t step, float step_size,
                           uint32_t k0, uint32_t k1, const McCvDev& cvk, cudaStream_t st) {
    const long long n = (long long)W * C;
    const int eb = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_mc_propose<<<eb, 256, 0, st>>>(s, sp, U, W, C, step, step_size, k0, k1, cvk);
}

void rid_launch_mc_accept_values(const float* aval, int na, int M, int W, int C, float* s, const float* sp, float* A,
                                 uint32_t step, float kT, uint32_t k0, uint32_t k1, int init, int count, int bins,
                                 int pi, int pj, unsigned long long* hist1, unsigned long long* hist2,
                                 unsigned long long* nacc, const McPathDev& path, const McCvDev& cvk,
                                 cudaStream_t st) {
    AcceptArgs a{};
    a.cvk = cvk;
    a.npath = path.n_nodes;
    a.Cp = path.n_cv;
    a.pcv = path.cv;
    a.pnodes = path.nodes;
    a.lam = path.lambda;
    a.z_lo = path.z_lo;
    a.z_hi = path.z_hi;
    a.histp = path.hist;
    a.aval = aval;
    a.na = na;
    a.M = M;
    a.W = W;
    a.C = C;
    a.s = s;
    a.sp = sp;
    a.A = A;
    a.step = step;
    a.k0 = k0;
    a.k1 = k1;
    a.kT = kT;
    a.init = init;
    a.count = count;
    a.bins = bins;
    a.pi = pi;
    a.pj = pj;
    a.hist1 = hist1;
    a.hist2 = hist2;
    a.nacc = nacc;
    const int wpb = 4;
    k_mc_accept<<<(W + wpb - 1) / wpb, 32 * wpb, 0, st>>>(a);
}

void rid_launch_mc_pmf(const unsigned long long* hist, int rows, int n, double kT, double* pmf, cudaStream_t st) {
    k_mc_pmf<<<rows, PT, 0, st>>>(hist, n, kT, pmf);
}
