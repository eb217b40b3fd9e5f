// k_select.cu -- the selection phase (Sec. "Selection phase": cluster_threshold,
// numb_cluster_lower / numb_cluster_upper, max_selection; Sec. "Selection":
// explored CVs are clustered and the values with high model deviation are
// collected by the trust levels; Sec. "CV selection": per-CV clustering
// weights and the angular mask).
//
//   k_sel_candidates  frames with trust_lo <= eps < trust_hi, compacted in
//                     frame order (one CTA, block-wide scans), CVs gathered
//   k_sel_leaders     leader clustering in candidate order: a candidate joins
//                     the first leader within the threshold, else it becomes a
//                     leader.  Candidates go in chunks of 1024, one per thread:
//                     each first checks the leaders of earlier chunks; one warp
//                     then settles the chunk's remaining candidates in order
//                     against the leaders this chunk created.  Same result as
//                     the sequential rule.
// The distance test decides integers, so it is taken in FP32 with explicitly
// rounded operations in a fixed order:
//   delta = a - b; periodic: delta -= 2 pi floor(delta / (2 pi) + 1/2);
//   d2 += w (delta delta); join iff d2 <= t^2 (t^2 rounded to FP32 once).
// The threshold search runs on the host (double), one clustering per trial.
#include <cmath>
#include <vector>

#include "rid_internal.cuh"

namespace {

constexpr int SEL_T = 1024;
constexpr float SEL_TWO_PI = 6.28318530717959f;
constexpr float SEL_INV_2PI = 0.159154943091895f;

__device__ __forceinline__ float sel_d2(const float* __restrict__ a, const float* __restrict__ b,
                                        const float* __restrict__ w, const int* __restrict__ per, int C) {
    float acc = 0.0f;
    for (int c = 0; c < C; ++c) {
        float d = __fsub_rn(a[c], b[c]);
        if (per[c]) {
            const float k = floorf(__fadd_rn(__fmul_rn(d, SEL_INV_2PI), 0.5f));
            d = __fsub_rn(d, __fmul_rn(SEL_TWO_PI, k));
        }
        acc = __fadd_rn(acc, __fmul_rn(w[c], __fmul_rn(d, d)));
    }
    return acc;
}

// Exclusive block scan of 0/1 flags over SEL_T threads; returns the prefix and
// writes the block total to *tot.
__device__ int block_excl_scan(int f, int* warp_sums, int* tot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int v = f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) warp_sums[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int s = warp_sums[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;   // inclusive over warps
        if (lane == 31) *tot = s;
    }
    __syncthreads();
    const int before = (wid ? warp_sums[wid - 1] : 0) + v - f;
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(SEL_T) k_sel_candidates(const float* __restrict__ cv, const float* __restrict__ eps,
                                                          int n, int C, float lo, float hi, int* __restrict__ cand,
                                                          float* __restrict__ ccv, int* __restrict__ n_cand) {
    __shared__ int warp_sums[32];
    __shared__ int tot;
    int base = 0;
    for (int c0 = 0; c0 < n; c0 += SEL_T) {
        const int k = c0 + threadIdx.x;
        const int f = (k < n && eps[k] >= lo && eps[k] < hi) ? 1 : 0;
        const int pos = block_excl_scan(f, warp_sums, &tot);
        if (f) cand[base + pos] = k;
        base += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_cand = base;
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)base * C; e += SEL_T) {
        const long long r = e / C;
        ccv[e] = cv[(long long)cand[r] * C + (e - r * C)];
    }
}

// leaders[] receives candidate row indices; *n_lead the count (or stop + 1
// when stop > 0 and the count passed it: the trial only needs "more than").
__global__ void __launch_bounds__(SEL_T) k_sel_leaders(const float* __restrict__ x, const int* __restrict__ n_cand_p,
                                                       int C, const float* __restrict__ w,
                                                       const int* __restrict__ per, float t2,
                                                       int* __restrict__ leaders, int* __restrict__ n_lead, int stop) {
    __shared__ int s_assign[SEL_T];
    __shared__ int s_nl;
    const int n = *n_cand_p;
    if (threadIdx.x == 0) s_nl = 0;
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += SEL_T) {
        const int k = c0 + threadIdx.x;
        const int nl0 = s_nl;
        int hit = -1;
        if (k < n) {
            const float* xk = x + (long long)k * C;
            for (int j = 0; j < nl0; ++j)
                if (sel_d2(x + (long long)leaders[j] * C, xk, w, per, C) <= t2) {
                    hit = j;
                    break;
                }
        }
        s_assign[threadIdx.x] = hit;
        __syncthreads();
        // settle the rest of the chunk in order against this chunk's new leaders
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            int nl = nl0;
            const int m = n - c0 < SEL_T ? n - c0 : SEL_T;
            for (int i = 0; i < m; ++i) {
                if (s_assign[i] >= 0) continue;
                const float* xi = x + (long long)(c0 + i) * C;
                bool found = false;
                for (int j0 = nl0; j0 < nl && !found; j0 += 32) {
                    const int j = j0 + lane;
                    const bool h = j < nl && sel_d2(x + (long long)leaders[j] * C, xi, w, per, C) <= t2;
                    found = __ballot_sync(0xffffffffu, h) != 0u;
                }
                if (!found) {
                    if (lane == 0) leaders[nl] = c0 + i;
                    ++nl;
                    __syncwarp();
                }
            }
            if (lane == 0) s_nl = nl;
        }
        __syncthreads();
        if (stop > 0 && s_nl > stop) break;
    }
    if (threadIdx.x == 0) *n_lead = s_nl;
}

// selected[i] = frame index of leader i (leaders hold candidate rows)
__global__ void k_sel_map(const int* __restrict__ lead, const int* __restrict__ cand, int n, int* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = cand[lead[i]];
}

int sel_cuda(cudaError_t e, const char* what) {
    return rid_fail(RID_ERR_CUDA, "select: %s: %s", what, cudaGetErrorString(e));
}

struct SelBuf {
    void* p = nullptr;
    ~SelBuf() {
        if (p) cudaFree(p);
    }
};

}  // namespace

extern "C" RID_API int rid_select(const rid_select_desc* d, int32_t n, const float* cv, const float* eps,
                                  int32_t* selected, int32_t* n_selected, int32_t* n_clusters, double* threshold_out,
                                  int32_t mem, void* stream) {
    NvtxScope nvtx_("rid_select");
    if (!d || !cv || !eps) return rid_fail(RID_ERR_ARG, "select: NULL argument");
    if (mem != RID_MEM_HOST && mem != RID_MEM_DEVICE) return rid_fail(RID_ERR_ARG, "select: bad mem");
    const int C = d->n_cv;
    if (C < 1 || C > RID_MAX_CV || n < 0 || !(d->cluster_threshold > 0) || d->max_selection < 0 ||
        (d->max_selection > 0 && !selected) ||
        (d->adapt && (d->numb_cluster_lower < 1 || d->numb_cluster_upper < d->numb_cluster_lower)))
        return rid_fail(RID_ERR_ARG, "select: parameters out of range");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<float> hw(C, 1.0f);
    std::vector<int> hp(C, 1);
    for (int c = 0; c < C; ++c) {
        if (d->weights) hw[c] = d->weights[c];
        if (d->periodic) hp[c] = d->periodic[c] != 0;
    }
    const long long nn = n > 0 ? n : 1;
    const size_t bytes = sizeof(float) * (size_t)(2 * nn * C + nn + C) + sizeof(int) * (size_t)(3 * nn + C + 2);
    SelBuf buf;
    if (cudaMalloc(&buf.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return rid_fail(RID_ERR_OOM, "select: device allocation of %zu bytes failed", bytes);
    }
    float* dcv = reinterpret_cast<float*>(buf.p);
    float* ccv = dcv + nn * C;
    float* deps = ccv + nn * C;
    float* dw = deps + nn;
    int* cand = reinterpret_cast<int*>(dw + C);
    int* lead = cand + nn;
    int* dper = lead + nn;
    int* dncand = dper + C;
    int* dnl = dncand + 1;
    int* dsel_buf = dnl + 1;   // [nn] frame indices of the selection
    const cudaMemcpyKind kin = mem == RID_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaError_t e;
    if (n > 0) {
        if ((e = cudaMemcpyAsync(dcv, cv, sizeof(float) * (size_t)n * C, kin, st)) != cudaSuccess) return sel_cuda(e, "cv");
        if ((e = cudaMemcpyAsync(deps, eps, sizeof(float) * (size_t)n, kin, st)) != cudaSuccess) return sel_cuda(e, "eps");
    }
    if ((e = cudaMemcpyAsync(dw, hw.data(), sizeof(float) * C, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return sel_cuda(e, "weights");
    if ((e = cudaMemcpyAsync(dper, hp.data(), sizeof(int) * C, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return sel_cuda(e, "mask");
    // trust window: eps in [lo, hi), compared in FP32 (the eps values are FP32)
    const float lo = (float)d->trust_lo, hi = (float)d->trust_hi;
    k_sel_candidates<<<1, SEL_T, 0, st>>>(dcv, deps, n, C, lo, hi, cand, ccv, dncand);
    int hn[2] = {0, 0};
    auto cluster = [&](double t, int stop, int* count) -> int {
        k_sel_leaders<<<1, SEL_T, 0, st>>>(ccv, dncand, C, dw, dper, (float)(t * t), lead, dnl, stop);
        cudaError_t e2;
        if ((e2 = cudaMemcpyAsync(hn, dncand, sizeof(int) * 2, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return sel_cuda(e2, "count");
        if ((e2 = cudaStreamSynchronize(st)) != cudaSuccess) return sel_cuda(e2, "synchronize");
        *count = hn[1];
        return RID_OK;
    };
    double t = d->cluster_threshold;
    int count = 0;
    // while searching, a clustering only needs to know whether its count passes
    // `upper`, so it stops there; the one finally kept is completed afterwards
    const int stop = d->adapt ? d->numb_cluster_upper : 0;
    if (int rc = cluster(t, stop, &count)) return rc;
    bool full = stop == 0 || count <= stop;   // the last clustering ran to the end
    if (d->adapt && hn[0] > 0) {
        const int lower = d->numb_cluster_lower, upper = d->numb_cluster_upper;
        double lo_t = 0.0, hi_t = INFINITY;
        for (int it = 0; it < 63; ++it) {
            if (count >= lower && count <= upper) break;
            if (count > upper) {
                lo_t = t;
                t = std::isinf(hi_t) ? 2.0 * t : std::sqrt(t * hi_t);
            } else {
                hi_t = t;
                t = lo_t == 0.0 ? 0.5 * t : std::sqrt(lo_t * t);
            }
            // a trial only needs to know whether the count passes `upper`
            if (int rc = cluster(t, upper, &count)) return rc;
            full = count <= upper;
        }
    }
    if (!full)
        if (int rc = cluster(t, 0, &count)) return rc;
    const int nsel = count < d->max_selection ? count : d->max_selection;
    if (nsel > 0) {
        int* dsel = mem == RID_MEM_DEVICE ? selected : dsel_buf;
        k_sel_map<<<(nsel + 255) / 256, 256, 0, st>>>(lead, cand, nsel, dsel);
        if ((e = cudaGetLastError()) != cudaSuccess) return sel_cuda(e, "map");
        if (mem == RID_MEM_HOST &&
            (e = cudaMemcpyAsync(selected, dsel, sizeof(int) * nsel, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return sel_cuda(e, "selected");
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return sel_cuda(e, "synchronize");
    }
    if (n_selected) *n_selected = nsel;
    if (n_clusters) *n_clusters = count;
    if (threshold_out) *threshold_out = t;
    return RID_OK;
}
