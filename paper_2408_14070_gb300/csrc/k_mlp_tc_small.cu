// k_mlp_tc_small.cu -- the tensor-core ensemble MLP (forward pass and input
// gradient) for small walker counts, with the GEMMs transposed.
//
// With few walkers a 128-row tile of k_mlp_tc is mostly empty, yet its
// epilogue turns a 128 x N accumulator into the next operand for every GEMM.
// Here each GEMM is computed as D^T = Wt . Act^T: the GEMM's outputs (neurons,
// or inputs in the backward pass) fill the MMA's M = 128 rows and the walkers,
// padded to NW = 16, 32 or 64, are its N columns.  The A operand is the same
// pre-swizzled weight image the other variants stream as their B operand --
// for GEMM g and 128-byte K-chunk c its rows are the GEMM's outputs, K-major
// -- so the same tensor maps load it, one 128-row M-tile per stage.  The B
// operand is the activation tile [walker][K] in the 128-byte swizzled K-major
// layout, NW rows per 64-column atom.
//
// TMEM: accumulator b of GEMM g holds M-tile mt in columns b * acc_cols +
// mt * NW .. + NW - 1; lane r of M-tile mt is output mt * 128 + r.  Epilogue
// warp w (w = 2..17) owns lane quarter w mod 4 and the M-tiles (w - 2) / 4,
// + 4, ...: a thread holds one output for NW walkers, reads them 16 columns at
// a time, and writes the next operand one BF16 value per walker.  The next
// GEMM's operand is released once per GEMM (every epilogue warp arrives on
// b_ready), after all of this GEMM's MMAs have completed, so a single operand
// buffer suffices.
//
// Per element the arithmetic is that of k_mlp_tc (bias, BF16 tanh, saved
// tanh in BF16, the FP32 residual stream, Delta = g (1 - t^2)); the member
// value A = w_out . h_L + b_out is reduced per (M-tile, lane quarter) by a
// warp butterfly and the partials added in a fixed order.  The MMA's operand
// roles are swapped, so its accumulation may round differently from the
// other variants: results agree with them within the BF16 bounds, not bit for
// bit, and the host selects this kernel by walker count alone (never by
// timing), so a given shape always gives the same bits.  A tcgen05.mma costs
// about the same whatever its N (measured: 60 MMAs of 128 x 16 x 16 take as
// long as 60 of 128 x 64 x 16, about 90 ns each, and interleaving M-tiles
// between K-steps made it slower), so the transposed form issues more MMAs
// per GEMM than the row form and wins only while its epilogue is much
// smaller: the host uses it for up to 16 walkers (NW = 16); the kernel also
// takes NW = 32 and 64.
// Scratch (per member, in the buffers the other variants use): saved tanh
// [L][Hp][NW] BF16 in tsave, the residual stream [Hp][NW] FP32 in rsave.
#include "rid_tc_ptx.cuh"

namespace {

constexpr int SM_MT = 4;     // M-tiles per GEMM (outputs up to 512)

struct SmemS {
    uint64_t full[TC_MAX_STAGES];
    uint64_t empty[TC_MAX_STAGES];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t b_ready;
    uint64_t drain;
    uint32_t tmem_base;
    int abort_flag;
};

// Byte offset of (walker row r, column col) in the activation operand: atoms
// of 64 BF16 columns x NW rows x 128 bytes, 16-byte chunk j of row r at
// position j ^ (r mod 8).
__device__ __forceinline__ uint32_t bs_off(int NW, int r, int col) {
    const int atom = col >> 6, ch = (col >> 3) & 7;
    return (uint32_t)atom * (uint32_t)(NW * 128) + (uint32_t)r * 128u + (uint32_t)((ch ^ (r & 7)) << 4) +
           (uint32_t)((col & 7) * 2);
}
__device__ __forceinline__ void st_bf16(unsigned char* B, uint32_t off, float v) {
    *reinterpret_cast<__nv_bfloat16*>(B + off) = __float2bfloat16_rn(v);
}
// tanh in BF16 of one value (the paired instruction on (x, x)), as a float
__device__ __forceinline__ float tanh_bf16(float x) {
    const uint32_t y = tanh_bf16x2(x, x);
    return __uint_as_float(y << 16);
}
// 32 lanes x 16 columns of TMEM into v[0..15]
__device__ __forceinline__ void tmem_ld16s(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <bool RES>
__global__ void __maxnreg__(96)
    k_mlp_tc_small(const __grid_constant__ TcArgs P, const __grid_constant__ CUtensorMap map_big,
                   const __grid_constant__ CUtensorMap map_small, int NW) {
    extern __shared__ __align__(1024) unsigned char dsm_raw[];
    unsigned char* dsm =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~uintptr_t(1023));
    __shared__ SmemS S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = blockIdx.y;
    const int L = P.L, G = P.ngemm, H = P.H;
    unsigned char* Bbuf = dsm;                                             // [Kpmax/64][NW rows][128 B]
    unsigned char* stages = dsm + (size_t)P.Kpmax * 2u * (size_t)NW;       // [NS][128 rows][128 B]
    const uint32_t stage_bytes = 128u * 128u;
    const int NS = P.stages;
    const int NACC = P.nacc;
    float* sbias = reinterpret_cast<float*>(stages + (size_t)NS * stage_bytes);   // [L][H]
    float* swout = sbias + (size_t)L * H;                                          // [H]
    float* spart = swout + H;                                                      // [SM_MT * 4][NW]
    volatile int* abort_flag = &S.abort_flag;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&S.full[s]), 1);
            mbar_init(smem_u32(&S.empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&S.acc_full[b]), 1);
            mbar_init(smem_u32(&S.acc_empty[b]), EPI_WARPS);
        }
        mbar_init(smem_u32(&S.b_ready), EPI_WARPS);
        mbar_init(smem_u32(&S.drain), 1);
        S.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"((uint32_t)P.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S.tmem_base;
    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer: weight M-tiles
        if (lane == 0) {
            int it = 0;
            int last_it[TC_MAX_STAGES];
            for (int s = 0; s < NS; ++s) last_it[s] = -1;
            bool ok = true;
            for (int g = 0; g < G && ok; ++g) {
                const int N = P.gN[g], nch = P.gKp[g] * 2 / 128, nm = (N + 127) / 128;
                for (int c = 0; c < nch && ok; ++c)
                    for (int mt = 0; mt < nm; ++mt, ++it) {
                        const int rows = N - mt * 128 < 128 ? N - mt * 128 : 128;
                        const int s = it % NS;
                        if (!mbar_wait(smem_u32(&S.empty[s]), ((it / NS) & 1) ^ 1, abort_flag, P.err, 1)) {
                            ok = false;
                            break;
                        }
                        mbar_arrive_tx(smem_u32(&S.full[s]), (uint32_t)rows * 128u);
                        last_it[s] = it;
                        const long long row0 = (long long)m * P.member_rows + P.grow[g] + (long long)c * N + mt * 128;
                        uint32_t dst = smem_u32(stages + (size_t)s * stage_bytes);
                        int r = 0;
                        for (; r + 64 <= rows; r += 64, dst += 8192u)
                            tma_load_2d(dst, &map_big, 0, (int)(row0 + r), smem_u32(&S.full[s]));
                        for (; r < rows; r += 8, dst += 1024u)
                            tma_load_2d(dst, &map_small, 0, (int)(row0 + r), smem_u32(&S.full[s]));
                    }
            }
            if (!ok) {
                for (int s = 0; s < NS; ++s)
                    if (last_it[s] >= 0) {
                        const unsigned long long t0 = gtimer();
                        while (!mbar_try(smem_u32(&S.full[s]), (last_it[s] / NS) & 1) && gtimer() - t0 < WAIT_NS) {}
                    }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer: M = 128 outputs, N = NW walkers
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            const uint32_t id = idesc_bf16(128, NW);
            for (int g = 0; g < G && ok; ++g) {
                const int N = P.gN[g], nch = P.gKp[g] * 2 / 128, nm = (N + 127) / 128;
                const int b = g % NACC;
                const uint32_t dacc = tmem + (uint32_t)(b * P.acc_cols);
                if (g >= NACC &&
                    !mbar_wait(smem_u32(&S.acc_empty[b]), ((g / NACC) - 1) & 1, abort_flag, P.err, 2)) {
                    ok = false;
                    break;
                }
                // the operand of GEMM g: written by the prologue (g = 0) or by GEMM g-1's epilogue
                if (!mbar_wait(smem_u32(&S.b_ready), g & 1, abort_flag, P.err, 4)) {
                    ok = false;
                    break;
                }
                fence_after();
                for (int c = 0; c < nch && ok; ++c) {
                    const uint32_t b_atom = smem_u32(Bbuf) + (uint32_t)(c * NW * 128);
                    for (int mt = 0; mt < nm; ++mt, ++it) {
                        const int s = it % NS;
                        if (!mbar_wait(smem_u32(&S.full[s]), (it / NS) & 1, abort_flag, P.err, 4)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        const uint32_t a_atom = smem_u32(stages + (size_t)s * stage_bytes);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma_bf16(dacc + (uint32_t)(mt * NW), desc_sw128(a_atom + 32u * kk),
                                     desc_sw128(b_atom + 32u * kk), id, (c | kk) != 0);
                        mma_commit(smem_u32(&S.empty[s]));
                    }
                }
                if (ok) mma_commit(smem_u32(&S.acc_full[b]));
            }
            mma_commit(smem_u32(&S.drain));
            const unsigned long long t0 = gtimer();
            while (!mbar_try(smem_u32(&S.drain), 0) && gtimer() - t0 < WAIT_NS) {}
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int e = warp - EPI_WARP0;          // 0..15
        const int quarter = warp & 3;            // TMEM lane quarter this warp may access
        const int sub = e >> 2;                  // first M-tile of this warp
        const int ET = 32 * EPI_WARPS;
        const int W = P.W;
        // GEMM 0 operand: u (FP32, [W][D]) -> [walker][K] BF16, zeros past D and for walkers >= W
        {
            const int kp0 = P.gKp[0];
            for (int it = e * 32 + lane; it < NW * (kp0 / 8); it += ET) {
                const int w = it % NW, col = (it / NW) * 8;
                float v[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int k = col + i;
                    v[i] = (w < W && k < P.D) ? __ldg(P.u + (size_t)w * P.D + k) : 0.0f;
                }
                *reinterpret_cast<uint4*>(Bbuf + bs_off(NW, w, col)) = pack8(v);
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&S.b_ready));
        }
        for (int idx = e * 32 + lane; idx < (L + 1) * H; idx += ET) {
            const int l = idx / H, c = idx - l * H;
            sbias[idx] = l < L ? __ldg(P.bias + ((size_t)m * L + l) * H + c) : __ldg(P.wout + (size_t)m * H + c);
        }
        asm volatile("bar.sync 1, %0;" ::"r"(ET) : "memory");   // all epilogue warps, before any bounded wait
        // per-member scratch: saved tanh [L][H][NW] BF16, residual stream [H][NW] FP32
        __nv_bfloat16* tsv = P.tsave + (size_t)m * P.ntiles * (size_t)L * 128 * H;
        float* rsv = RES ? P.rsave + (size_t)m * P.ntiles * (size_t)128 * H : nullptr;
        for (int g = 0; g < G; ++g) {
            const int N = P.gN[g], nm = (N + 127) / 128;
            const bool fwd = g < L;
            const int l = fwd ? g : (2 * L - 1 - g);
            const int b = g % NACC;
            const int kpn = g + 1 < G ? P.gKp[g + 1] : 0;   // the next GEMM's K: columns N .. kpn - 1 are zero
            const bool res_fwd = RES && fwd && l >= 1;
            const bool res_bwd = RES && !fwd && l >= 1;
            const bool res_st = RES && (fwd ? l < L - 1 : l >= 2);
            if (!mbar_wait(smem_u32(&S.acc_full[b]), (g / NACC) & 1, abort_flag, P.err, 8)) break;
            fence_after();
            for (int mt = sub; mt < nm; mt += 4) {
                const int n = mt * 128 + quarter * 32 + lane;   // the output this thread holds
                const bool vn = n < N;
                const uint32_t tacc = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * P.acc_cols + mt * NW);
                const float bn = (fwd && vn) ? sbias[l * H + n] : 0.0f;
                const float wo = vn && n < H ? swout[n] : 0.0f;
                for (int w0 = 0; w0 < NW; w0 += 16) {
                    float a[16];
                    tmem_ld16s(tacc + (uint32_t)w0, a);
                    // the residual stream of this output for the 16 walkers, read whole
                    // before any of it is overwritten
                    float rp[16];
                    float4* rq = RES ? reinterpret_cast<float4*>(rsv + (size_t)n * NW + w0) : nullptr;
                    if (RES && vn && (res_fwd || (res_bwd && l < L - 1))) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float4 v = rq[q];
                            rp[4 * q] = v.x;
                            rp[4 * q + 1] = v.y;
                            rp[4 * q + 2] = v.z;
                            rp[4 * q + 3] = v.w;
                        }
                    }
                    tmem_wait_ld();
                    float out[16];   // this GEMM's contribution to the next operand
                    float part[16];  // member value terms w_out[n] h_L[n][w] (last forward layer)
                    float rs[16];    // residual stream values to store
                    if (fwd) {
                        __nv_bfloat16 tb[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const float t = tanh_bf16(a[i] + bn);
                            tb[i] = __float2bfloat16_rn(t);
                            float h = t;
                            if (RES && res_fwd && vn) h = rp[i] + t;
                            rs[i] = h;
                            part[i] = vn ? wo * h : 0.0f;
                            out[i] = l == L - 1 ? wo * (1.0f - t * t) : h;
                        }
                        if (vn) {
                            uint4* dst = reinterpret_cast<uint4*>(tsv + ((size_t)l * H + n) * NW + w0);
                            dst[0] = *reinterpret_cast<const uint4*>(&tb[0]);
                            dst[1] = *reinterpret_cast<const uint4*>(&tb[8]);
                        }
                    } else if (l > 0) {
                        // G_{l-1} (+ dA/dh_l) -> Delta_{l-1} = G (1 - t_{l-1}^2)
                        __nv_bfloat16 tb[16];
                        if (vn) {
                            const uint4* src = reinterpret_cast<const uint4*>(tsv + ((size_t)(l - 1) * H + n) * NW + w0);
                            *reinterpret_cast<uint4*>(&tb[0]) = src[0];
                            *reinterpret_cast<uint4*>(&tb[8]) = src[1];
                        }
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            float gv = a[i];
                            if (RES && res_bwd && vn) gv = (l == L - 1 ? wo : rp[i]) + gv;
                            rs[i] = gv;
                            const float t = vn ? __bfloat162float(tb[i]) : 0.0f;
                            out[i] = gv * (1.0f - t * t);
                            part[i] = 0.0f;
                        }
                    } else {
                        // G_0 = dA/du (n is an input index): dA/ds_j = -sin s_j g[2j] + cos s_j g[2j+1]
                        // (torsion), g[2j] (distance); the pair's odd element comes from the next lane
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const float g1 = __shfl_down_sync(0xffffffffu, a[i], 1);
                            const int w = w0 + i, j = n >> 1;
                            if (!(n & 1) && 2 * j < P.D && w < W && !*abort_flag) {
                                const float cs = __ldg(P.u + (size_t)w * P.D + 2 * j);
                                const float sn = __ldg(P.u + (size_t)w * P.D + 2 * j + 1);
                                const bool dist = P.cvdist && __ldg(P.cvdist + j);
                                P.gradA[((size_t)m * W + w) * P.C + j] = dist ? a[i] : -sn * a[i] + cs * g1;
                            }
                            out[i] = 0.0f;
                            part[i] = 0.0f;
                            rs[i] = 0.0f;
                        }
                    }
                    if (RES && res_st && vn) {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            rq[q] = make_float4(rs[4 * q], rs[4 * q + 1], rs[4 * q + 2], rs[4 * q + 3]);
                    }
                    if (g < G - 1 && n < kpn) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) st_bf16(Bbuf, bs_off(NW, w0 + i, n), vn ? out[i] : 0.0f);
                    }
                    if (fwd && l == L - 1) {
                        // member value: this warp's 32 outputs, butterfly over the lanes
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            float p = part[i];
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
                            if (lane == 0) spart[(mt * 4 + quarter) * NW + w0 + i] = p;
                        }
                    }
                }
            }
            if (g < G - 1) {
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&S.b_ready));
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&S.acc_empty[b]));
        }
    }
    fence_before();
    __syncthreads();
    // member value A = sum over (M-tile, lane quarter) partials in that order, + b_out
    if (warp >= EPI_WARP0 && warp < EPI_WARP0 + 2) {
        const int w = (warp - EPI_WARP0) * 32 + lane;
        const int nmL = (P.gN[L - 1] + 127) / 128;
        if (w < P.W && w < NW && !S.abort_flag) {
            float a = 0.0f;
            for (int q = 0; q < nmL * 4; ++q) a += spart[q * NW + w];
            P.Apart[(size_t)m * P.W + w] = a + __ldg(P.bout + m);
        }
    }
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)P.tmem_cols)
                     : "memory");
    }
}

}  // namespace

size_t rid_mlp_tc_small_smem_bytes(const TcArgs& P, int NW) {
    return 1024 + (size_t)P.Kpmax * 2u * NW + (size_t)P.stages * 128u * 128u +
           sizeof(float) * ((size_t)(P.L + 1) * P.H + (size_t)SM_MT * 4 * NW);
}

cudaError_t rid_launch_mlp_tc_small(const TcArgs& P, const CUtensorMap& big, const CUtensorMap& small, int NW,
                                    cudaStream_t s) {
    if (P.ngemm != 2 * P.L || P.W > NW || (NW != 16 && NW != 32 && NW != 64)) return cudaErrorInvalidValue;
    if (P.resnet && !P.rsave) return cudaErrorInvalidValue;
    if (P.geb[0] != 2) return cudaErrorInvalidValue;   // BF16 only
    const size_t smem = rid_mlp_tc_small_smem_bytes(P, NW);
    const int v = P.resnet ? 1 : 0;
    static size_t attr[2][64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    size_t& have = attr[v][dev & 63];
    auto kern = v == 0 ? k_mlp_tc_small<false> : k_mlp_tc_small<true>;
    if (smem > have) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        have = smem;
    }
    kern<<<dim3(1, P.M, 1), NTHREADS, smem, s>>>(P, big, small, NW);
    return cudaGetLastError();
}
