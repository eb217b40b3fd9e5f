// rid_tc_ptx.cuh -- inline-PTX helpers of the tcgen05 ensemble kernels:
// bounded mbarrier waits, shared-memory matrix and instruction descriptors,
// tcgen05 MMA / commit / TMEM loads, tensor TMA loads, and the BF16 / FP8
// packing of operand tiles in the 128-byte swizzled K-major layout.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "rid_internal.cuh"
#include "rid_tc.cuh"

namespace {

constexpr int EPI_WARP0 = 2;
constexpr int EPI_WARPS = 16;                       // 4 per TMEM lane quarter
constexpr int NTHREADS = 32 * (EPI_WARP0 + EPI_WARPS);
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

// tcgen05 shared-memory matrix descriptor for a K-major operand in the
// 128-byte swizzled layout: start >> 4, leading byte offset 16 (unused for
// this layout), stride byte offset 1024 (between 8-row groups), version 1 at
// bit 46, layout type 2 (128-byte swizzle) at bits 61-63.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
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
__device__ __forceinline__ uint32_t idesc_e4m3(int M, int N) {
    // kind::f8f6f4 instruction descriptor: D F32 (bit 4), A and B E4M3 (format
    // code 0 in bits 7-9 and 10-12), K-major A and B, N >> 3 at bit 17, M >> 4 at bit 24
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_e4m3(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p; }" ::"r"(d),
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
// tanh of two values rounded to BF16, result packed as BF16x2 (the operand
// and scratch format); hardware approximation with BF16 output precision.
__device__ __forceinline__ uint32_t tanh_bf16x2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    uint32_t x = *reinterpret_cast<uint32_t*>(&h), y;
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ uint4 pack8(const float (&v)[8]) {
    return make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
}
__device__ __forceinline__ void unpack_bf16x8(uint4 w, float (&v)[8]) {
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        v[2 * i] = __uint_as_float(u[i] << 16);
        v[2 * i + 1] = __uint_as_float(u[i] & 0xFFFF0000u);
    }
}
// Two floats -> two FP8 e4m3 bytes, x in the low byte (round to nearest even,
// saturating at +-448).
__device__ __forceinline__ uint32_t pack_e4m3x2(float x, float y) {
    uint16_t r;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(y), "f"(x));
    return r;
}
__device__ __forceinline__ uint2 pack8_e4m3(const float (&v)[8]) {
    return make_uint2(pack_e4m3x2(v[0], v[1]) | (pack_e4m3x2(v[2], v[3]) << 16),
                      pack_e4m3x2(v[4], v[5]) | (pack_e4m3x2(v[6], v[7]) << 16));
}
// Element offset of (layer l, row, 8-column group starting at col) in a
// tile's saved-tanh scratch [L][H/8][128][8]: the 32 rows of a warp touch one
// contiguous 512-byte line.
__device__ __forceinline__ size_t ts_off(int l, int row, int col, int H) {
    return (((size_t)l * (H / 8) + (col >> 3)) * 128 + row) * 8;
}
// Byte offset of (row, column col; col a multiple of 8) in the 128-row
// swizzled A tile: 64-column atoms of 128 rows x 128 bytes.
__device__ __forceinline__ uint32_t a_off(int row, int col) {
    const int atom = col >> 6, ch = (col >> 3) & 7;
    return (uint32_t)atom * (128u * 128u) + (uint32_t)row * 128u + (uint32_t)((ch ^ (row & 7)) << 4);
}

// Byte offset of (row, column col; col a multiple of 8) in the FP8 A tile:
// 128-column atoms, 16 columns per 16-byte chunk.
__device__ __forceinline__ uint32_t a_off8(int row, int col) {
    const int atom = col >> 7, ch = (col >> 4) & 7;
    return (uint32_t)atom * (128u * 128u) + (uint32_t)row * 128u + (uint32_t)((ch ^ (row & 7)) << 4) +
           (uint32_t)(col & 8);
}
// Eight A-operand values of one row at columns col..col+7 in the operand
// format of the GEMM that reads them (eb bytes per element).
__device__ __forceinline__ void store_a8(unsigned char* A, int row, int col, int eb, const float (&v)[8]) {
    if (eb == 2) *reinterpret_cast<uint4*>(A + a_off(row, col)) = pack8(v);
    else *reinterpret_cast<uint2*>(A + a_off8(row, col)) = pack8_e4m3(v);
}
__device__ __forceinline__ void zero_a8(unsigned char* A, int row, int col, int eb) {
    if (eb == 2) *reinterpret_cast<uint4*>(A + a_off(row, col)) = make_uint4(0, 0, 0, 0);
    else *reinterpret_cast<uint2*>(A + a_off8(row, col)) = make_uint2(0, 0);
}

// Member value A = w_out . h_L + b_out from the partial sums of 16-column
// slices (each an FMA chain over its columns from zero), added in column
// order: the same bits whichever CTA computed which slice.
__device__ __forceinline__ size_t qs_off(int m, int tile, int slice, int row, int ntiles) {
    return (((size_t)m * ntiles + tile) * TC_MAX_QSLICES + slice) * 128 + row;
}
__device__ __forceinline__ float member_value(const TcArgs& P, int m, int tile, int row) {
    float a = 0.0f;
    for (int q = 0; q < P.H / 16; ++q) a += P.qsave[qs_off(m, tile, q, row, P.ntiles)];
    return a + __ldg(P.bout + m);
}

}  // namespace

// ---------------------------------------------------------------------------
// Thread-block cluster helpers (distributed shared memory).
namespace {

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster_v4(uint32_t a, uint4 v) {
    asm volatile("st.shared::cluster.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}
__device__ __forceinline__ void st_cluster_v2(uint32_t a, uint2 v) {
    asm volatile("st.shared::cluster.v2.b32 [%0], {%1, %2};" ::"r"(a), "r"(v.x), "r"(v.y) : "memory");
}
__device__ __forceinline__ void st_cluster_f32(uint32_t a, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
// Arrive on an mbarrier of CTA `rank` (release at cluster scope).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t local_bar, uint32_t rank) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(mapa(local_bar, rank))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_cluster(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on a barrier that other CTAs of the cluster arrive on.
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t a, uint32_t parity, volatile int* abort_flag, int* err,
                                                  int code) {
    if (mbar_try_cluster(a, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (true) {
        if (mbar_try_cluster(a, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > WAIT_NS) {
            *abort_flag = 1;
            atomicOr(err, code);
            return false;
        }
    }
}
__device__ __forceinline__ void fence_async_smem_cluster() {
    asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
}
// Arrive on a local mbarrier and raise its expected transaction bytes.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(a), "r"(bytes)
                 : "memory");
}
// Bulk copy of `bytes` (a multiple of 16) from this CTA's shared memory to the
// same offset in CTA `rank`, completing on that CTA's mbarrier (complete_tx).
__device__ __forceinline__ void bulk_copy_to_peer(uint32_t local_src, uint32_t bytes, uint32_t local_bar,
                                                  uint32_t rank) {
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            mapa(local_src, rank)),
        "r"(local_src), "r"(bytes), "r"(mapa(local_bar, rank))
        : "memory");
}
__device__ __forceinline__ void bulk_commit_and_wait_read() {
    asm volatile("cp.async.bulk.commit_group;\n\tcp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

}  // namespace
