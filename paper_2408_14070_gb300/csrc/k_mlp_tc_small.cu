// k_mlp_tc_small.cu -- the tensor-core ensemble MLP (forward pass and input
// gradient) for small walker counts, with the GEMMs transposed and each
// GEMM's 128-output tiles split over a thread-block cluster.
//
// With few walkers a 128-row tile of k_mlp_tc is mostly empty, yet its
// epilogue turns a 128 x N accumulator into the next operand for every GEMM.
// Here each GEMM is computed as D^T = Wt . Act^T: the GEMM's outputs (neurons,
// or inputs in the backward pass) fill the MMA's M = 128 rows and the walkers,
// padded to NW = 16, are its N columns.  The A operand is the same
// pre-swizzled weight image the other variants stream as their B operand --
// for GEMM g and 128-byte K-chunk c its rows are the GEMM's outputs, K-major
// -- so the same tensor maps load it, one 128-row M-tile per stage.  The B
// operand is the activation tile [walker][K] in the 128-byte swizzled K-major
// layout, NW rows per 64-column atom.
//
// Cluster split: a cluster of CS CTAs (1..4) serves one member; CTA rank r
// owns the M-tiles mt = r, r + CS, ... of every GEMM (local tile j = mt / CS),
// streams only their weight rows and issues only their MMAs.  The outputs of
// tile mt are columns [128 mt, 128 mt + 128) of the next GEMM's operand: two
// whole 64-column atoms, one contiguous block of NW x 256 bytes.  The
// epilogue writes them into this CTA's operand buffer and a copy warp sends
// the block to every peer that owns tiles of the next GEMM with one bulk
// shared-to-shared copy, completing on the peer's barrier of received bytes
// (its MMA warp raises the barrier's expected bytes by what the peers send).
// The operand is double buffered (GEMM g reads buffer g mod 2), so a copy for
// GEMM g + 1 never lands in a buffer a peer's GEMM g still reads.  A tcgen05
// .mma costs about 90-115 ns whatever its N (measured), so the split divides
// the chain's MMA time by CS.
//
// Every tile accumulates its K-chunks in order; a CTA waits for the received
// bytes only before its first chunk from a peer (rank 0 starts on its own).
// Every M-tile is accumulated by the same sequence of MMAs whichever CTA owns
// it, and the member value is added in a fixed order on rank 0, so every
// cluster size gives the same bits.  Measured and not kept: starting each
// tile on the chunks its own CTA wrote (a rotated K order: every MMA became
// slower, 42 -> 49 us for the paper's network at 12 walkers), and even and odd
// K-steps in two accumulators added in the epilogue (slower too).
//
// TMEM: accumulator b of GEMM g holds local tile j in columns b * acc_cols +
// j * NW .. + NW - 1; lane r of tile mt is output 128 mt + r.  Epilogue warp w
// owns lane quarter w mod 4 and the 4-walker groups (w - 2) / 4 (+ E / 4) of
// every local tile.  Per element
// the arithmetic is that of k_mlp_tc (bias, BF16 tanh, saved tanh in BF16, the
// FP32 residual stream, Delta = g (1 - t^2)); the member value A = w_out . h_L
// + b_out is reduced per (M-tile, lane quarter) by a warp butterfly and the
// partials added in a fixed order.  The MMA's operand roles are swapped, so
// its accumulation may round differently from the row variants: results
// agree with them within the BF16 bounds, not bit for bit, and the host
// selects this kernel by walker count alone (never by timing).
//
// The saved tanh [L][rows][NW] BF16 and the residual stream [rows][NW] FP32 of
// a CTA's own outputs stay in its shared memory: the backward pass reads
// exactly the outputs the same CTA produced in the forward pass (the backward
// GEMM of layer l has layer l - 1's neurons as outputs, tiled the same way).
// Both are stored in 4-walker chunks with the chunk index XOR-swizzled by
// row, so that a warp's 32 consecutive rows hit distinct banks.
//
// Warp roles: warp 0 TMA producer, warp 1 TMEM allocator and MMA issuer,
// warps 2..2+E-1 epilogue (E = 16, or 8 in the lean variant, whose warps each
// take two 4-walker groups: 352 threads instead of 608, so that with few
// weight stages a CTA can share an SM with other kernels' CTAs), warp 2+E bulk
// copies of the exchange.  Every wait is
// bounded in time; a CTA whose wait expires sets the error word and stops
// issuing, its peers' waits then expire too, and every CTA still meets the
// final cluster barrier, so no CTA exits while another may write into it.
#include <algorithm>

#include "rid_tc_ptx.cuh"

namespace {

constexpr int SM_MT = 4;                       // M-tiles per GEMM (outputs up to 512)
constexpr int SM_GRP = 4;                      // walkers per epilogue work item
// threads of a CTA with `epi` epilogue warps (16, or 8 for the lean variant)
constexpr int sm_threads(int epi) { return 32 * (EPI_WARP0 + epi + 1); }

constexpr int NW = 16;                         // MMA columns: walkers padded to 16

struct SmemS {
    uint64_t full[TC_MAX_STAGES];
    uint64_t empty[TC_MAX_STAGES];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t b_local[2];      // this CTA's chunks of operand buffer b written: 16 epilogue warps
    uint64_t b_peer[2];       // the peers' chunks of buffer b received: the MMA warp's expect-tx arrival
                              // and the peers' bytes
    uint64_t slice_done[2];   // this CTA's chunks of the operand in buffer b written: 16 epilogue warps
    uint64_t drain;
    uint32_t tmem_base;
    int abort_flag;
};

// Byte offset of (walker row r, column col) in the activation operand: atoms
// of 64 BF16 columns x 16 rows x 128 bytes, 16-byte chunk j of row r at
// position j ^ (r mod 8).
__device__ __forceinline__ uint32_t bs_off(int r, int col) {
    const int atom = col >> 6, ch = (col >> 3) & 7;
    return (uint32_t)atom * (uint32_t)(NW * 128) + (uint32_t)r * 128u + (uint32_t)((ch ^ (r & 7)) << 4) +
           (uint32_t)((col & 7) * 2);
}
__device__ __forceinline__ void st_bf16(unsigned char* B, uint32_t off, float v) {
    *reinterpret_cast<__nv_bfloat16*>(B + off) = __float2bfloat16_rn(v);
}
// Residual stream: local output row, 4-walker chunk cg, as a float4 index.
// Two rows share a 128-byte line (8 chunks); the chunk is XOR-ed with the
// row's pair index so that 8 consecutive rows hit 8 distinct chunk slots.
__device__ __forceinline__ int rs_idx(int row, int cg) { return row * 4 + (cg ^ ((row >> 1) & 3)); }
// Saved tanh: layer l, local row, 4-walker chunk cg (8 bytes), as a uint2
// index.  Four rows share a 128-byte line (16 slots of 8 bytes).
__device__ __forceinline__ int ts_idx(int rows, int l, int row, int cg) {
    return (l * rows + row) * 4 + (cg ^ ((row >> 2) & 3));
}
// 32 lanes x 4 columns of TMEM
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
// M-tiles of GEMM g owned by rank r of CS (mt = r + j CS < nm)
__device__ __forceinline__ int owned_tiles(int nm, int r, int CS) { return r < nm ? (nm - r + CS - 1) / CS : 0; }
// Atoms [a0, a1) of the next operand written by tile mt (kpn: the next GEMM's K)
__device__ __forceinline__ void tile_atoms(int mt, int kpn, int& a0, int& a1) {
    a0 = 2 * mt;
    a1 = 2 * mt + 2 < kpn / 64 ? 2 * mt + 2 : kpn / 64;
}
// Bytes of GEMM g's operand (g >= 1) that CTA `rank` receives from its peers
__device__ __forceinline__ uint32_t peer_bytes(const TcArgs& P, int g, int rank, int CS) {
    const int kp = P.gKp[g], nmp = (P.gN[g - 1] + 127) / 128;
    int own = 0;
    for (int mt = rank; mt < nmp; mt += CS) {
        int a0, a1;
        tile_atoms(mt, kp, a0, a1);
        own += a1 - a0;
    }
    return (uint32_t)(kp / 64 - own) * (uint32_t)NW * 128u;
}
// Is K-chunk c of GEMM g's operand (g >= 1) written by this CTA?  Chunk c
// comes from tile c / 2 of GEMM g - 1.
__device__ __forceinline__ bool own_chunk(int c, int rank, int CS) { return (c >> 1) % CS == rank; }

// 608 threads x 96 registers at 16 epilogue warps (a launch with 104 asks for too many)
template <bool RES, int EPI>
__global__ void __maxnreg__(96)
    k_mlp_tc_small(const __grid_constant__ TcArgs P, const __grid_constant__ CUtensorMap map_big,
                   const __grid_constant__ CUtensorMap map_small) {
    extern __shared__ __align__(1024) unsigned char dsm_raw[];
    unsigned char* dsm =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~uintptr_t(1023));
    __shared__ SmemS S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int CS = P.csize;
    const int rank = (int)cluster_rank();
    const int m = blockIdx.y;
    const int L = P.L, G = P.ngemm, H = P.H;
    int nmx = 1;
    for (int g = 0; g < G; ++g) nmx = max(nmx, (P.gN[g] + 127) / 128);
    const int rows = owned_tiles(nmx, 0, CS) * 128;                        // local output rows (rank 0 owns most)
    const size_t bbytes = (size_t)P.Kpmax * 2u * (size_t)NW;
    // operand buffers 0 and 1, [Kp/64][16 rows][128 B] each
    auto Bbuf = [&](int i) -> unsigned char* { return dsm + (size_t)i * bbytes; };
    unsigned char* stages = dsm + 2 * bbytes;                               // [NS][128 rows][128 B]
    const uint32_t stage_bytes = 128u * 128u;
    const int NS = P.stages;
    const int NACC = P.nacc;
    uint2* tsv = reinterpret_cast<uint2*>(stages + (size_t)NS * stage_bytes);             // [L][rows][4]
    float4* rsv = reinterpret_cast<float4*>(tsv + (size_t)L * rows * 4);                  // [rows][4] (RES)
    float* sbias = reinterpret_cast<float*>(rsv + (RES ? (size_t)rows * 4 : 0));          // [L][H]
    float* swout = sbias + (size_t)L * H;                                                  // [H]
    float* spart = swout + H;                                                              // [SM_MT * 4][NW]
    volatile int* abort_flag = &S.abort_flag;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&S.full[s]), 1);
            mbar_init(smem_u32(&S.empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&S.acc_full[b]), 1);
            mbar_init(smem_u32(&S.acc_empty[b]), EPI);
            mbar_init(smem_u32(&S.b_local[b]), EPI);
            mbar_init(smem_u32(&S.b_peer[b]), 1);
            mbar_init(smem_u32(&S.slice_done[b]), EPI);
        }
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
    // barriers initialised in every CTA before any peer copies into them
    cluster_sync_all();
    fence_after();
    const uint32_t tmem = S.tmem_base;
    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer: this CTA's weight M-tiles
        if (lane == 0) {
            int it = 0;
            int last_it[TC_MAX_STAGES];
            for (int s = 0; s < NS; ++s) last_it[s] = -1;
            bool ok = true;
            for (int g = 0; g < G && ok; ++g) {
                const int N = P.gN[g], nch = P.gKp[g] * 2 / 128;
                const int nj = owned_tiles((N + 127) / 128, rank, CS);
                for (int c = 0; c < nch && ok; ++c)
                    for (int j = 0; j < nj; ++j, ++it) {
                        const int mt = rank + j * CS;
                        const int rws = N - mt * 128 < 128 ? N - mt * 128 : 128;
                        const int s = it % NS;
                        if (!mbar_wait(smem_u32(&S.empty[s]), ((it / NS) & 1) ^ 1, abort_flag, P.err, 1)) {
                            ok = false;
                            break;
                        }
                        mbar_arrive_tx(smem_u32(&S.full[s]), (uint32_t)rws * 128u);
                        last_it[s] = it;
                        const long long row0 = (long long)m * P.member_rows + P.grow[g] + (long long)c * N + mt * 128;
                        uint32_t dst = smem_u32(stages + (size_t)s * stage_bytes);
                        int r = 0;
                        for (; r + 64 <= rws; r += 64, dst += 8192u)
                            tma_load_2d(dst, &map_big, 0, (int)(row0 + r), smem_u32(&S.full[s]));
                        for (; r < rws; r += 8, dst += 1024u)
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
        // ------------------------------------------------------------ MMA issuer: M = 128 outputs, N = 16 walkers
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            const uint32_t id = idesc_bf16(128, NW);
            for (int g = 0; g < G && ok; ++g) {
                const int N = P.gN[g], nch = P.gKp[g] * 2 / 128, nm = (N + 127) / 128;
                const int nj = owned_tiles(nm, rank, CS);
                const int b = g % NACC;
                const uint32_t dacc = tmem + (uint32_t)(b * P.acc_cols);
                if (g >= NACC &&
                    !mbar_wait(smem_u32(&S.acc_empty[b]), ((g / NACC) - 1) & 1, abort_flag, P.err, 2)) {
                    ok = false;
                    break;
                }
                // the operand of GEMM g: the prologue (g = 0) or GEMM g-1's epilogues; this CTA's
                // chunks written locally, the peers' chunks arriving as bytes on b_peer
                const uint32_t pb = (g > 0 && rank < nm) ? peer_bytes(P, g, rank, CS) : 0u;
                mbar_arrive_expect_tx(smem_u32(&S.b_peer[g & 1]), pb);
                if (!mbar_wait(smem_u32(&S.b_local[g & 1]), (g >> 1) & 1, abort_flag, P.err, 4)) {
                    ok = false;
                    break;
                }
                fence_after();
                bool have_peer = false;
                const uint32_t bbase = smem_u32(Bbuf(g & 1));
                for (int c = 0; c < nch && ok; ++c) {
                    if (!have_peer && g > 0 && !own_chunk(c, rank, CS)) {
                        if (!mbar_wait_cluster(smem_u32(&S.b_peer[g & 1]), (g >> 1) & 1, abort_flag, P.err, 4)) {
                            ok = false;
                            break;
                        }
                        have_peer = true;
                        fence_after();
                    }
                    const uint32_t b_atom = bbase + (uint32_t)(c * NW * 128);
                    for (int j = 0; j < nj; ++j, ++it) {
                        const int s = it % NS;
                        if (!mbar_wait(smem_u32(&S.full[s]), (it / NS) & 1, abort_flag, P.err, 4)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        const uint32_t a_atom = smem_u32(stages + (size_t)s * stage_bytes);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma_bf16(dacc + (uint32_t)(j * NW), desc_sw128(a_atom + 32u * kk),
                                     desc_sw128(b_atom + 32u * kk), id, (c | kk) != 0);
                        mma_commit(smem_u32(&S.empty[s]));
                    }
                }
                // every phase of b_peer is waited on, so that no peer's copy is still landing at exit
                if (ok && !have_peer &&
                    !mbar_wait_cluster(smem_u32(&S.b_peer[g & 1]), (g >> 1) & 1, abort_flag, P.err, 4))
                    ok = false;
                if (ok) mma_commit(smem_u32(&S.acc_full[b]));
            }
            mma_commit(smem_u32(&S.drain));
            const unsigned long long t0 = gtimer();
            while (!mbar_try(smem_u32(&S.drain), 0) && gtimer() - t0 < WAIT_NS) {}
        }
    } else if (warp == EPI_WARP0 + EPI) {
        // ------------------------------------------------------------ bulk exchange
        if (lane == 0 && CS > 1) {
            for (int g = 0; g + 1 < G; ++g) {
                if (!mbar_wait(smem_u32(&S.slice_done[g & 1]), (g >> 1) & 1, abort_flag, P.err, 16)) break;
                const int nm = (P.gN[g] + 127) / 128, kpn = P.gKp[g + 1];
                const int nmn = (P.gN[g + 1] + 127) / 128;   // peers owning tiles of GEMM g+1 need the operand
                const int nq = CS < nmn ? CS : nmn;
                for (int mt = rank; mt < nm; mt += CS) {
                    int a0, a1;
                    tile_atoms(mt, kpn, a0, a1);
                    if (a1 <= a0) continue;
                    const uint32_t bytes = (uint32_t)(a1 - a0) * (uint32_t)NW * 128u;
                    const uint32_t src = smem_u32(Bbuf((g + 1) & 1)) + (uint32_t)a0 * (uint32_t)NW * 128u;
                    for (int q = 0; q < nq; ++q)
                        if (q != rank) bulk_copy_to_peer(src, bytes, smem_u32(&S.b_peer[(g + 1) & 1]), (uint32_t)q);
                }
                bulk_commit_and_wait_read();
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int e = warp - EPI_WARP0;          // 0..EPI-1
        const int quarter = warp & 3;            // TMEM lane quarter this warp may access
        const int sub = e >> 2;                  // this warp's first 4-walker group
        const int ET = 32 * EPI;
        const int W = P.W;
        const int q32 = quarter * 32 + lane;     // the row within a tile this thread holds
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
                *reinterpret_cast<uint4*>(Bbuf(0) + bs_off(w, col)) = pack8(v);
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&S.b_local[0]));
        }
        for (int idx = e * 32 + lane; idx < (L + 1) * H; idx += ET) {
            const int l = idx / H, c = idx - l * H;
            sbias[idx] = l < L ? __ldg(P.bias + ((size_t)m * L + l) * H + c) : __ldg(P.wout + (size_t)m * H + c);
        }
        asm volatile("bar.sync 1, %0;" ::"r"(ET) : "memory");   // all epilogue warps, before any bounded wait
        for (int g = 0; g < G; ++g) {
            const int N = P.gN[g], nm = (N + 127) / 128;
            const int nj = owned_tiles(nm, rank, CS);
            const bool fwd = g < L;
            const int l = fwd ? g : (2 * L - 1 - g);
            const int b = g % NACC;
            const int kpn = g + 1 < G ? P.gKp[g + 1] : 0;   // the next GEMM's K: columns N .. kpn - 1 are zero
            const bool res_fwd = RES && fwd && l >= 1;
            const bool res_bwd = RES && !fwd && l >= 1;
            const bool res_st = RES && (fwd ? l < L - 1 : l >= 2);
            const bool res_ld = res_fwd || (res_bwd && l < L - 1);
            unsigned char* Bn = Bbuf((g + 1) & 1);
            if (!mbar_wait(smem_u32(&S.acc_full[b]), (g / NACC) & 1, abort_flag, P.err, 8)) break;
            fence_after();
            // this warp's 4 walkers of the local tiles, two tiles loaded before each wait
            // the warp's 4-walker groups cg = sub, sub + EPI / 4, ...
#pragma unroll 1
            for (int cg = sub; cg < NW / SM_GRP; cg += EPI / 4) {
                const uint32_t tq = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * P.acc_cols + cg * SM_GRP);
#pragma unroll 1
                for (int j0 = 0; j0 < nj; j0 += 2) {
                    float a[2][SM_GRP];
                    tmem_ld4(tq + (uint32_t)(j0 * NW), a[0]);
                    if (j0 + 1 < nj) tmem_ld4(tq + (uint32_t)((j0 + 1) * NW), a[1]);
                    tmem_wait_ld();
#pragma unroll
                    for (int jj = 0; jj < 2; ++jj) {
                        const int j = j0 + jj;
                        if (j >= nj) break;
                        const int mt = rank + j * CS;
                        const int row = j * 128 + q32;          // local output row
                        const int n = mt * 128 + q32;           // the output this thread holds
                        const bool vn = n < N;
                        const float bn = (fwd && vn) ? sbias[l * H + n] : 0.0f;
                        const float wo = vn && n < H ? swout[n] : 0.0f;
                        float rp[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                        if (RES && vn && res_ld) {
                            const float4 v = rsv[rs_idx(row, cg)];
                            rp[0] = v.x;
                            rp[1] = v.y;
                            rp[2] = v.z;
                            rp[3] = v.w;
                        }
                        float out[4];    // this GEMM's contribution to the next operand
                        float part[4];   // member value terms w_out[n] h_L[n][w] (last forward layer)
                        float rs[4];     // residual stream values to store
                        if (fwd) {
                            // t = tanh(z) in BF16, elementwise on pairs of walkers
                            const uint32_t y01 = tanh_bf16x2(a[jj][0] + bn, a[jj][1] + bn);
                            const uint32_t y23 = tanh_bf16x2(a[jj][2] + bn, a[jj][3] + bn);
                            const float t[4] = {__uint_as_float(y01 << 16), __uint_as_float(y01 & 0xffff0000u),
                                                __uint_as_float(y23 << 16), __uint_as_float(y23 & 0xffff0000u)};
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                float h = t[i];
                                if (RES && res_fwd && vn) h = rp[i] + t[i];
                                rs[i] = h;
                                part[i] = vn ? wo * h : 0.0f;
                                out[i] = l == L - 1 ? wo * (1.0f - t[i] * t[i]) : h;
                            }
                            if (vn) tsv[ts_idx(rows, l, row, cg)] = make_uint2(y01, y23);
                        } else if (l > 0) {
                            // G_{l-1} (+ dA/dh_l) -> Delta_{l-1} = G (1 - t_{l-1}^2)
                            const uint2 tw = vn ? tsv[ts_idx(rows, l - 1, row, cg)] : make_uint2(0u, 0u);
                            const float t[4] = {__uint_as_float(tw.x << 16), __uint_as_float(tw.x & 0xffff0000u),
                                                __uint_as_float(tw.y << 16), __uint_as_float(tw.y & 0xffff0000u)};
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                float gv = a[jj][i];
                                if (RES && res_bwd && vn) gv = (l == L - 1 ? wo : rp[i]) + gv;
                                rs[i] = gv;
                                out[i] = gv * (1.0f - t[i] * t[i]);
                                part[i] = 0.0f;
                            }
                        } else {
                            // G_0 = dA/du (n is an input index): dA/ds_j = -sin s_j g[2j] + cos s_j g[2j+1]
                            // (torsion), g[2j] (distance); the pair's odd element comes from the next lane
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const float g1 = __shfl_down_sync(0xffffffffu, a[jj][i], 1);
                                const int w = cg * SM_GRP + i, jc = n >> 1;
                                if (!(n & 1) && 2 * jc < P.D && w < W && !*abort_flag) {
                                    const float cs = __ldg(P.u + (size_t)w * P.D + 2 * jc);
                                    const float sn = __ldg(P.u + (size_t)w * P.D + 2 * jc + 1);
                                    const bool dist = P.cvdist && __ldg(P.cvdist + jc);
                                    P.gradA[((size_t)m * W + w) * P.C + jc] = dist ? a[jj][i] : -sn * a[jj][i] + cs * g1;
                                }
                                out[i] = 0.0f;
                                part[i] = 0.0f;
                                rs[i] = 0.0f;
                            }
                        }
                        if (RES && res_st && vn) rsv[rs_idx(row, cg)] = make_float4(rs[0], rs[1], rs[2], rs[3]);
                        if (g < G - 1 && n < kpn) {
                            const int ch = (n >> 3) & 7;
                            const uint32_t cb = (uint32_t)(n >> 6) * (uint32_t)(NW * 128) + (uint32_t)((n & 7) * 2);
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                st_bf16(Bn, cb + (uint32_t)(cg * SM_GRP + i) * 128u + (uint32_t)((ch ^ ((cg * SM_GRP + i) & 7)) << 4),
                                        vn ? out[i] : 0.0f);
                        }
                        if (fwd && l == L - 1) {
                            // member value: this warp's 32 outputs, butterfly over the lanes, into rank 0
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                float p = part[i];
#pragma unroll
                                for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
                                if (lane == 0)
                                    st_cluster_f32(mapa(smem_u32(&spart[(mt * 4 + quarter) * NW + cg * SM_GRP + i]), 0u), p);
                            }
                        }
                    }
                }
            }
            if (g < G - 1) {
                fence_async_smem();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(smem_u32(&S.b_local[(g + 1) & 1]));
                    if (CS > 1) mbar_arrive(smem_u32(&S.slice_done[g & 1]));
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&S.acc_empty[b]));
        }
    }
    fence_before();
    __syncthreads();
    // every CTA's partials are in rank 0: member value A = sum over (M-tile, lane quarter)
    // in that order, + b_out
    cluster_sync_all();
    if (rank == 0 && warp >= EPI_WARP0 && warp < EPI_WARP0 + 2) {
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

// Shared memory of the small-batch kernel at P.csize CTAs per member and
// P.stages weight stages (0: the fixed part alone).
size_t rid_mlp_tc_small_smem_bytes(const TcArgs& P, int nw) {
    int nmx = 1;
    for (int g = 0; g < 2 * P.L; ++g) nmx = std::max(nmx, (P.gN[g] + 127) / 128);
    const int CS = P.csize < 1 ? 1 : P.csize;
    const size_t rows = (size_t)((nmx + CS - 1) / CS) * 128;
    return 1024 + 2 * (size_t)P.Kpmax * 2u * nw + (size_t)P.stages * 128u * 128u + (size_t)P.L * rows * nw * 2u +
           (P.resnet ? rows * nw * 4u : 0) + sizeof(float) * ((size_t)(P.L + 1) * P.H + (size_t)SM_MT * 4 * nw);
}

cudaError_t rid_launch_mlp_tc_small(const TcArgs& P, const CUtensorMap& big, const CUtensorMap& small, int nw,
                                    int epi_warps, cudaStream_t s) {
    if (P.ngemm != 2 * P.L || P.W > NW || nw != NW) return cudaErrorInvalidValue;
    if (P.csize < 1 || P.csize > SM_MT || P.stages < 2 || P.stages > TC_MAX_STAGES) return cudaErrorInvalidValue;
    if (epi_warps != 16 && epi_warps != 8) return cudaErrorInvalidValue;
    if (P.geb[0] != 2) return cudaErrorInvalidValue;   // BF16 only
    for (int g = 0; g < 2 * P.L; ++g)
        if (P.gN[g] > 128 * SM_MT) return cudaErrorInvalidValue;
    const size_t smem = rid_mlp_tc_small_smem_bytes(P, NW);
    const int v = (P.resnet ? 1 : 0) + (epi_warps == 8 ? 2 : 0);
    static size_t attr[4][64] = {};   // shared memory opted into, per instantiation and device
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    size_t& have = attr[v][dev & 63];
    auto kern = v == 0 ? k_mlp_tc_small<false, 16> : v == 1 ? k_mlp_tc_small<true, 16>
              : v == 2 ? k_mlp_tc_small<false, 8> : k_mlp_tc_small<true, 8>;
    if (smem > have) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        have = smem;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(P.csize, P.M, 1);
    cfg.blockDim = dim3(sm_threads(epi_warps), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = P.csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, P, big, small);
}
