// k_mlp_tc.cu -- BF16 ensemble MLP on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in TMEM, weights streamed by tensor TMA).
//
// Work unit: one tile of 128 walkers x one ensemble member, split over a
// cluster of CS CTAs (CS = 1, 2 or 4); CTA rank q computes output neurons
// [q N/CS, (q+1) N/CS) of every layer.  For each member the chain of 2L GEMMs
//   forward  l = 0..L-1 :  Z_l = H_{l-1} W_l^T      (128 x H,   K = D' or H)
//   backward l = L-1..0 :  G_{l-1} = Delta_l W_l     (128 x fin, K = H)
// runs with the activation tile (A operand, BF16, canonical no-swizzle
// K-major layout) in shared memory and the weight slice (B operand) streamed
// in K-chunks through a ring of TMA stages.  Epilogues (8 warps) read the
// FP32 accumulator from TMEM, apply bias + tanh (forward) or the tanh
// derivative (backward), write the next A operand, and for CS > 1 copy their
// column slice to every peer CTA's A buffer with DSMEM bulk copies.
//   g_L = w_out, Delta_l = g_l * (1 - tanh^2 z_l), g_{l-1} = W_l^T Delta_l,
//   dA/ds_j = -sin s_j g_0[2j] + cos s_j g_0[2j+1].
// tanh(z_l) is kept as BF16 in a global scratch for the backward pass.
//
// Warp roles (320 threads): warp 0 = TMA producer, warp 1 = TMEM allocator +
// MMA issuer, warps 2..9 = epilogue (two warps per TMEM lane quarter, each
// with half of the columns).  Every wait is bounded in time; a wait that
// expires sets an error word, drains the copies and MMAs already issued and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include "rid_internal.cuh"
#include "rid_tc.cuh"

namespace {

constexpr int NTHREADS = 320;
constexpr int EPI_WARP0 = 2;
constexpr unsigned long long WAIT_NS = 1000000000ull;   // 1 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t a, uint32_t bytes) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(a), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false if the deadline passed or another role aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag, int* err, int code) {
    if (mbar_try(a, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (true) {
        if (mbar_try(a, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > WAIT_NS) {
            *abort_flag = 1;
            atomicOr(err, code);
            return false;
        }
    }
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    // tcgen05 shared-memory matrix descriptor, no swizzle, K-major operand:
    // start >> 4 | LBO >> 4 << 16 | SBO >> 4 << 32 | version 1 << 46
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
    // kind::f16 instruction descriptor: D F32 (bit 4), A BF16 (bits 7-9 = 1),
    // B BF16 (bits 10-12 = 1), K-major A and B, N >> 3 at bit 17, M >> 4 at bit 24
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t mapa(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void dsmem_bulk(uint32_t dst_cluster, uint32_t src, uint32_t bytes, uint32_t bar_cluster) {
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst_cluster),
        "r"(src), "r"(bytes), "r"(bar_cluster)
        : "memory");
}
__device__ __forceinline__ float tanh_fast(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ void unpack_bf16x8(uint4 w, float (&v)[8]) {
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        v[2 * i] = __uint_as_float(u[i] << 16);
        v[2 * i + 1] = __uint_as_float(u[i] & 0xFFFF0000u);
    }
}

struct Smem {
    uint64_t full[TC_MAX_STAGES];
    uint64_t empty[TC_MAX_STAGES];
    uint64_t acc_full;
    uint64_t a_full[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort_flag;
    float apart[2][128];
};

__global__ void __launch_bounds__(NTHREADS, 1)
    k_mlp_tc(const __grid_constant__ TcArgs P, const __grid_constant__ CUtensorMap map_big,
             const __grid_constant__ CUtensorMap map_small) {
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ Smem S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int CS = P.CS;
    const uint32_t q = CS > 1 ? cluster_rank() : 0u;
    const int tile = blockIdx.x / CS, m = blockIdx.y;
    const int L = P.L, G = 2 * L;
    const int Kmax = P.Kmax;
    const uint32_t abytes = 128u * (uint32_t)Kmax * 2u;
    unsigned char* Abuf[2] = {dsm, dsm + (CS > 1 ? abytes : 0u)};
    unsigned char* stages = dsm + (CS > 1 ? 2u : 1u) * abytes;
    const uint32_t stage_bytes = P.stage_bytes;
    const int NS = P.stages;
    volatile int* abort_flag = &S.abort_flag;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&S.full[s]), 1);
            mbar_init(smem_u32(&S.empty[s]), 1);
        }
        mbar_init(smem_u32(&S.acc_full), 1);
        mbar_init(smem_u32(&S.a_full[0]), 8);
        mbar_init(smem_u32(&S.a_full[1]), 8);
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
    if (CS > 1) cluster_sync();
    else __syncthreads();
    fence_after();
    const uint32_t tmem = S.tmem_base;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            int it = 0;
            int last_it[TC_MAX_STAGES];
            for (int s = 0; s < NS; ++s) last_it[s] = -1;
            bool ok = true;
            for (int g = 0; g < G && ok; ++g) {
                const int N = P.gN[g], K = P.gK[g], ns = N / CS;
                const int nch = K / P.ck;
                const uint32_t bytes = (uint32_t)ns * P.ck * 2u;
                const int rows = (int)(bytes / 128u);
                for (int c = 0; c < nch; ++c, ++it) {
                    const int s = it % NS;
                    if (!mbar_wait(smem_u32(&S.empty[s]), ((it / NS) & 1) ^ 1, abort_flag, P.err, 1)) { ok = false; break; }
                    mbar_arrive_tx(smem_u32(&S.full[s]), bytes);
                    last_it[s] = it;
                    const long long row0 = (long long)m * P.member_rows + P.grow[g] + (long long)(c * CS + (int)q) * rows;
                    uint32_t dst = smem_u32(stages + (size_t)s * stage_bytes);
                    int r = 0;
                    for (; r + 64 <= rows; r += 64, dst += 8192u)
                        tma_load_2d(dst, &map_big, 0, (int)(row0 + r), smem_u32(&S.full[s]));
                    for (; r < rows; r += 8, dst += 1024u)
                        tma_load_2d(dst, &map_small, 0, (int)(row0 + r), smem_u32(&S.full[s]));
                }
            }
            if (!ok) {
                // let the loads already issued land before the CTA can exit
                for (int s = 0; s < NS; ++s)
                    if (last_it[s] >= 0) {
                        const unsigned long long t0 = gtimer();
                        while (!mbar_try(smem_u32(&S.full[s]), (last_it[s] / NS) & 1) && gtimer() - t0 < WAIT_NS) {}
                    }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            int issued = 0;
            for (int g = 0; g < G && ok; ++g) {
                const int N = P.gN[g], K = P.gK[g], ns = N / CS;
                const int nch = K / P.ck;
                const int b = CS > 1 ? (g & 1) : 0;
                const uint32_t apar = CS > 1 ? ((g >> 1) & 1) : (g & 1);
                if (!mbar_wait(smem_u32(&S.a_full[b]), apar, abort_flag, P.err, 2)) { ok = false; break; }
                fence_after();
                const uint32_t abase = smem_u32(Abuf[b]);
                const uint32_t id = idesc_bf16(128, ns < 256 ? ns : 256);
                for (int c = 0; c < nch; ++c, ++it) {
                    const int s = it % NS;
                    if (!mbar_wait(smem_u32(&S.full[s]), (it / NS) & 1, abort_flag, P.err, 4)) { ok = false; break; }
                    fence_after();
                    const uint32_t bbase = smem_u32(stages + (size_t)s * stage_bytes);
                    for (int kk = 0; kk < P.ck / 16; ++kk) {
                        const int k0 = c * P.ck + kk * 16;   // first K index of this MMA
                        // A: k-block stride 128 rows x 16 B = 2048 B, 8-row group stride 128 B
                        const uint64_t ad = smem_desc(abase + (uint32_t)(k0 / 8) * 2048u, 2048u, 128u);
                        // B slice: k-block stride ns/8 x 128 B, 8-row group stride 128 B
                        for (int n0 = 0; n0 < ns; n0 += 256) {
                            // rows n0.. of the slice start n0/8 row groups (128 B each) further
                            const uint64_t bd = smem_desc(bbase + (uint32_t)(kk * 2) * (uint32_t)ns * 16u +
                                                              (uint32_t)(n0 / 8) * 128u,
                                                          (uint32_t)ns * 16u, 128u);
                            mma_bf16(tmem + (uint32_t)n0, ad, bd, ns - n0 >= 256 ? id : idesc_bf16(128, ns - n0),
                                     (c | kk) != 0);
                            ++issued;
                        }
                    }
                    mma_commit(smem_u32(&S.empty[s]));
                }
                if (ok) mma_commit(smem_u32(&S.acc_full));
            }
            // every MMA issued has completed before TMEM can be released
            mma_commit(smem_u32(&S.drain));
            const unsigned long long t0 = gtimer();
            while (!mbar_try(smem_u32(&S.drain), 0) && gtimer() - t0 < WAIT_NS) {}
            (void)issued;
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int e = warp - EPI_WARP0;          // 0..7
        const int quarter = warp & 3;            // TMEM lane quarter this warp may access
        const int half = e >> 2;                 // column half
        const int row = quarter * 32 + lane;     // walker within the tile
        const int wg = tile * 128 + row;         // global walker
        const bool valid = wg < P.W;
        const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
        const int nsf = P.H / CS;                // this CTA's forward column slice
        float* sbias = reinterpret_cast<float*>(stages + (size_t)NS * stage_bytes);   // [L][nsf]
        float* swout = sbias + (size_t)L * nsf;                                        // [nsf]
        // per-CTA copies of the biases / output weights of this column slice
        for (int idx = e * 32 + lane; idx < (L + 1) * nsf; idx += 256) {
            const int l = idx / nsf, c = idx - l * nsf;
            const int gc = (int)q * nsf + c;
            sbias[idx] = l < L ? __ldg(P.bias + ((size_t)m * L + l) * P.H + gc) : __ldg(P.wout + (size_t)m * P.H + gc);
        }
        // GEMM 0 input: u (FP32, [W][D]) -> BF16 canonical tile, all Dp columns
        {
            unsigned char* A0 = Abuf[0];
            const int ngroups = P.Dp / 8;
            for (int kb = half; kb < ngroups; kb += 2) {
                float v[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int k = kb * 8 + i;
                    v[i] = (valid && k < P.D) ? __ldg(P.u + (size_t)wg * P.D + k) : 0.0f;
                }
                uint4 w4 = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                      pack_bf16(v[6], v[7]));
                *reinterpret_cast<uint4*>(A0 + (size_t)kb * 2048 + row * 16) = w4;
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&S.a_full[0]));
        }
        asm volatile("bar.sync 1, 256;" ::: "memory");   // staged biases visible to all epilogue warps
        __nv_bfloat16* tsave_tile = P.tsave + ((size_t)m * P.ntiles + tile) * (size_t)L * 128 * P.H;
        float apart = 0.0f;
        for (int g = 0; g < G; ++g) {
            const int N = P.gN[g], ns = N / CS;
            const int col0 = (int)q * ns;              // global column of local column 0
            const int ngr = ns / 8, gh = ngr / 2;      // 8-column groups, per half
            const int gbeg = half * gh, gend = gbeg + gh;
            const bool fwd = g < L;
            const int l = fwd ? g : (G - 1 - g);       // layer of this GEMM
            unsigned char* Anext = Abuf[CS > 1 ? ((g + 1) & 1) : 0];
            // prefetch the saved tanh values of the first batch (independent of the accumulator)
            uint4 tpre[4];
            if (!fwd && l > 0) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (gbeg + k < gend)
                        tpre[k] = *reinterpret_cast<const uint4*>(tsave_tile + ((size_t)(l - 1) * 128 + row) * P.H +
                                                                   col0 + (gbeg + k) * 8);
            }
            if (CS > 1 && g >= 1 && lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
            __syncwarp();
            if (!mbar_wait(smem_u32(&S.acc_full), g & 1, abort_flag, P.err, 8)) break;
            fence_after();
            for (int gb = gbeg; gb < gend; gb += 4) {
                const int nb = gend - gb < 4 ? gend - gb : 4;
                float acc[4][8];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (k < nb) tmem_ld8(trow + (uint32_t)((gb + k) * 8), acc[k]);
                if (!fwd && l > 0 && gb != gbeg) {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (k < nb)
                            tpre[k] = *reinterpret_cast<const uint4*>(tsave_tile + ((size_t)(l - 1) * 128 + row) * P.H +
                                                                       col0 + (gb + k) * 8);
                }
                tmem_wait_ld();
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (k >= nb) break;
                    const int gi = gb + k;
                    const int gc = col0 + gi * 8;          // global column of this group
                    const int lc = gi * 8;                 // column within this CTA's slice
                    if (fwd) {
                        const float* bias = sbias + (size_t)l * nsf + lc;
                        float t[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) t[i] = tanh_fast(acc[k][i] + bias[i]);
                        uint4 tw = make_uint4(pack_bf16(t[0], t[1]), pack_bf16(t[2], t[3]), pack_bf16(t[4], t[5]),
                                              pack_bf16(t[6], t[7]));
                        *reinterpret_cast<uint4*>(tsave_tile + ((size_t)l * 128 + row) * P.H + gc) = tw;
                        uint4 ow;
                        if (l == L - 1) {
                            const float* wo = swout + lc;
                            float d[8];
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                apart = fmaf(wo[i], t[i], apart);
                                d[i] = wo[i] * (1.0f - t[i] * t[i]);
                            }
                            ow = make_uint4(pack_bf16(d[0], d[1]), pack_bf16(d[2], d[3]), pack_bf16(d[4], d[5]),
                                            pack_bf16(d[6], d[7]));
                        } else {
                            ow = tw;
                        }
                        *reinterpret_cast<uint4*>(Anext + (size_t)(gc / 8) * 2048 + row * 16) = ow;
                    } else if (l > 0) {
                        // G_{l-1} -> Delta_{l-1} = G (1 - t_{l-1}^2)
                        float t[8], d[8];
                        unpack_bf16x8(tpre[k], t);
#pragma unroll
                        for (int i = 0; i < 8; ++i) d[i] = acc[k][i] * (1.0f - t[i] * t[i]);
                        *reinterpret_cast<uint4*>(Anext + (size_t)(gc / 8) * 2048 + row * 16) =
                            make_uint4(pack_bf16(d[0], d[1]), pack_bf16(d[2], d[3]), pack_bf16(d[4], d[5]),
                                       pack_bf16(d[6], d[7]));
                    } else if (valid) {
                        // G_0 = dA/du: dA/ds_j = -sin s_j g[2j] + cos s_j g[2j+1]
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            const int j = gc / 2 + p;
                            if (2 * j < P.D) {
                                const float cs = __ldg(P.u + (size_t)wg * P.D + 2 * j);
                                const float sn = __ldg(P.u + (size_t)wg * P.D + 2 * j + 1);
                                P.gradA[((size_t)m * P.W + wg) * P.C + j] = -sn * acc[k][2 * p] + cs * acc[k][2 * p + 1];
                            }
                        }
                    }
                }
            }
            if (fwd && l == L - 1) S.apart[half][row] = apart;
            fence_before();
            if (g == G - 1) break;
            fence_async_smem();
            __syncwarp();
            const int b = CS > 1 ? ((g + 1) & 1) : 0;
            if (lane == 0) {
                if (CS > 1) {
                    // this warp's 32 rows of each of its column groups -> every peer's buffer
                    for (int gi = gbeg; gi < gend; ++gi) {
                        const uint32_t src = smem_u32(Anext + (size_t)((col0 + gi * 8) / 8) * 2048 + quarter * 512);
                        for (int p = 1; p < CS; ++p) {
                            const uint32_t peer = (q + (uint32_t)p) % (uint32_t)CS;
                            dsmem_bulk(mapa(src, peer), src, 512u, mapa(smem_u32(&S.a_full[b]), peer));
                        }
                    }
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                }
                if (e == 0 && CS > 1) mbar_arrive_tx(smem_u32(&S.a_full[b]), (uint32_t)(CS - 1) * (uint32_t)ns * 256u);
                else mbar_arrive(smem_u32(&S.a_full[b]));
            }
        }
        if (CS > 1 && lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    // member value A = w_out . h_L + b_out (this CTA's column slice)
    if (warp >= EPI_WARP0 && warp < EPI_WARP0 + 4) {
        const int row = (warp & 3) * 32 + lane;
        const int wg = tile * 128 + row;
        if (wg < P.W && !S.abort_flag) {
            float a = S.apart[0][row] + S.apart[1][row];
            if (q == 0) a += __ldg(P.bout + m);
            P.Apart[((size_t)m * CS + q) * P.W + wg] = a;
        }
    }
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)P.tmem_cols)
                     : "memory");
    }
    if (CS > 1) cluster_sync();
}

}  // namespace

size_t rid_mlp_tc_smem_bytes(const TcArgs& P) {
    const size_t abytes = 128u * (size_t)P.Kmax * 2u;
    return (P.CS > 1 ? 2 : 1) * abytes + (size_t)P.stages * P.stage_bytes +
           sizeof(float) * (size_t)(P.L + 1) * (P.H / P.CS);
}

cudaError_t rid_launch_mlp_tc(const TcArgs& P, const CUtensorMap& big, const CUtensorMap& small, cudaStream_t s) {
    const size_t smem = rid_mlp_tc_smem_bytes(P);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (P.CS > 1) {
        e = cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P.ntiles * P.CS, P.M, 1);
    cfg.blockDim = dim3(NTHREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = P.CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_mlp_tc, P, big, small);
}
