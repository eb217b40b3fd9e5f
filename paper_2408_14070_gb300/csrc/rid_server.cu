// rid_server.cu -- the server object: a budgeted device memory pool, pinned
// staging, and batched restrained labeling through the persistent kernel
// k_label_fused (one launch for any number of uneven jobs), with a timing
// autotuner for the kernel's CTA size.
#include <algorithm>
#include <cstdarg>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>

#include "rid_batch.cuh"

#define SCK(call)                                                                                           \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess)                                                                              \
            return rid_fail(e_ == cudaErrorMemoryAllocation ? RID_ERR_OOM : RID_ERR_CUDA, "%s: %s (%s:%d)", \
                            #call, cudaGetErrorString(e_), __FILE__, __LINE__);                             \
    } while (0)

#define STRY(expr)                      \
    do {                                \
        const int r_ = (expr);          \
        if (r_ != RID_OK) return r_;    \
    } while (0)

namespace {

constexpr size_t POOL_ALIGN = 256;
constexpr size_t LF_SMEM_LIMIT = 220 * 1024;

inline size_t align_up(size_t n) { return (n + POOL_ALIGN - 1) & ~(POOL_ALIGN - 1); }

// First-fit allocator over one device allocation of the server's budget.
// Free blocks are kept by offset and merged with their neighbours on release.
class Pool {
  public:
    int init(size_t bytes) {
        cudaError_t e = cudaMalloc(&base_, bytes);
        if (e != cudaSuccess) {
            base_ = nullptr;
            cudaGetLastError();
            return rid_fail(RID_ERR_OOM, "rid_server_create: cudaMalloc(%zu) failed: %s", bytes,
                            cudaGetErrorString(e));
        }
        cap_ = bytes;
        free_.clear();
        free_[0] = bytes;
        used_ = 0;
        return RID_OK;
    }
    void release() {
        if (base_) cudaFree(base_);
        base_ = nullptr;
        free_.clear();
        cap_ = used_ = 0;
    }
    // Offset of n bytes (256-byte aligned), or SIZE_MAX if no block fits.
    size_t alloc(size_t n) {
        n = align_up(n ? n : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const size_t off = it->first, rest = it->second - n;
            free_.erase(it);
            if (rest) free_[off + n] = rest;
            used_ += n;
            return off;
        }
        return SIZE_MAX;
    }
    void free(size_t off, size_t n) {
        n = align_up(n ? n : 1);
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    char* base() const { return static_cast<char*>(base_); }
    size_t used() const { return used_; }
    size_t capacity() const { return cap_; }

  private:
    void* base_ = nullptr;
    size_t cap_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;
};

// Grow-only pinned host buffer.
struct Pinned {
    void* p = nullptr;
    size_t bytes = 0;
    int ensure(size_t n) {
        if (n <= bytes) return RID_OK;
        if (p) cudaFreeHost(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaHostAlloc(&p, n, cudaHostAllocDefault);
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            return rid_fail(RID_ERR_OOM, "cudaHostAlloc(%zu) failed: %s", n, cudaGetErrorString(e));
        }
        bytes = n;
        return RID_OK;
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = nullptr;
        bytes = 0;
    }
    char* c() const { return static_cast<char*>(p); }
};

// Device bytes of one label job and where its arrays sit in its region.  The
// label accumulators and flags are contiguous so one descriptor zeroes them.
struct JobLayout {
    size_t x, v, f, s0, kappa, mf, se, sd, sum, sum2, bsum, flags, zero_bytes, bytes;
};

JobLayout job_layout(int R, int N, int C, int B) {
    JobLayout L{};
    size_t o = 0;
    auto put = [&](size_t n) { const size_t at = o; o = align_up(o + n); return at; };
    const size_t nb = (size_t)R * N, nc = (size_t)R * C;
    L.x = put(16 * nb);
    L.v = put(16 * nb);
    L.f = put(16 * nb);
    L.s0 = put(8 * nc);
    L.kappa = put(8 * nc);
    L.mf = put(8 * nc);
    L.se = put(8 * nc);
    L.sd = put(8 * nc);
    L.sum = o;
    o += 8 * nc;
    L.sum2 = o;
    o += 8 * nc;
    L.bsum = o;
    o += 8 * nc * (size_t)B;
    L.flags = o;
    o += 4 * (size_t)R;
    L.zero_bytes = o - L.sum;
    L.bytes = align_up(o);
    return L;
}

}  // namespace

// ---------------------------------------------------------------------------
struct rid_server {
    int device = 0, n_sm = 0;
    Pool pool;
    Pinned pin_in, pin_out, pin_meta;
    void* d_meta = nullptr;       // job table, items, descriptors, counter (grow-only, outside the budget)
    size_t d_meta_bytes = 0;
    std::map<long long, int> tuned;   // batch-shape key -> CTA size
    int last_threads = 0;
};

namespace {

int ensure_meta(rid_server* srv, size_t n) {
    if (n <= srv->d_meta_bytes) return RID_OK;
    if (srv->d_meta) cudaFree(srv->d_meta);
    srv->d_meta = nullptr;
    srv->d_meta_bytes = 0;
    cudaError_t e = cudaMalloc(&srv->d_meta, n);
    if (e != cudaSuccess) {
        srv->d_meta = nullptr;
        cudaGetLastError();
        return rid_fail(RID_ERR_OOM, "cudaMalloc(%zu) for batch tables failed", n);
    }
    srv->d_meta_bytes = n;
    return RID_OK;
}

int check_server_device(rid_server* srv) {
    int dev = -1;
    SCK(cudaGetDevice(&dev));
    if (dev != srv->device)
        return rid_fail(RID_ERR_STATE, "server was created on device %d, current device is %d", srv->device, dev);
    return RID_OK;
}

// Validation shared by the batch call: the limits of rid_label plus the
// persistent kernel's shared-memory limit.
int check_label_job(const rid_label_job& j, int idx, int device) {
    if (!j.sys || !j.x0 || !j.s0 || !j.kappa || !j.mf_out || !j.se_out || !j.std_out)
        return rid_fail(RID_ERR_ARG, "job %d: NULL argument", idx);
    if (rid_sys_device(j.sys) != device)
        return rid_fail(RID_ERR_STATE, "job %d: system lives on device %d, server on %d", idx, rid_sys_device(j.sys),
                        device);
    if (j.n_runs < 1) return rid_fail(RID_ERR_ARG, "job %d: n_runs=%d must be >= 1", idx, j.n_runs);
    if (j.n_blocks < 2 || j.n_blocks > RID_MAX_BLOCKS)
        return rid_fail(RID_ERR_ARG, "job %d: n_blocks=%d outside [2, %d]", idx, j.n_blocks, RID_MAX_BLOCKS);
    if (j.n_equil < 0 || j.n_steps - j.n_equil < j.n_blocks)
        return rid_fail(RID_ERR_ARG, "job %d: need 0 <= n_equil and n_steps - n_equil >= n_blocks", idx);
    if (j.step0 + (uint64_t)j.n_steps > (1ull << 32))
        return rid_fail(RID_ERR_ARG, "job %d: step0 + n_steps exceeds 2^32", idx);
    const SysDev* S = rid_sys_dev(j.sys);
    if (rid_label_fused_smem(S->N, S->C, 0) > LF_SMEM_LIMIT)
        return rid_fail(RID_ERR_ARG, "job %d: a chain of %d beads and %d CVs needs %zu bytes of shared memory (> %zu)",
                        idx, S->N, S->C, rid_label_fused_smem(S->N, S->C, 0), LF_SMEM_LIMIT);
    return RID_OK;
}

long long shape_key(int n_items, int maxN) {
    int a = 0, b = 0;
    while ((1 << a) < n_items && a < 30) ++a;
    while ((1 << b) < maxN && b < 30) ++b;
    return (long long)a * 64 + b;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" int rid_server_create(uint64_t budget, rid_server** out) {
    if (!out) return rid_fail(RID_ERR_ARG, "NULL out");
    *out = nullptr;
    if (budget < (1u << 20)) return rid_fail(RID_ERR_ARG, "hbm_budget_bytes=%llu below 1 MiB", (unsigned long long)budget);
    rid_server* srv = new rid_server();
    cudaError_t e = cudaGetDevice(&srv->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&srv->n_sm, cudaDevAttrMultiProcessorCount, srv->device);
    if (e != cudaSuccess) {
        delete srv;
        return rid_fail(RID_ERR_CUDA, "rid_server_create: %s", cudaGetErrorString(e));
    }
    const int rc = srv->pool.init((size_t)budget);
    if (rc != RID_OK) {
        delete srv;
        return rc;
    }
    *out = srv;
    return RID_OK;
}

extern "C" int rid_server_destroy(rid_server* srv) {
    if (!srv) return RID_OK;
    cudaDeviceSynchronize();
    srv->pool.release();
    srv->pin_in.release();
    srv->pin_out.release();
    srv->pin_meta.release();
    if (srv->d_meta) cudaFree(srv->d_meta);
    delete srv;
    return RID_OK;
}

extern "C" int rid_label_batch(rid_server* srv, const rid_label_job* jobs, int32_t n_jobs, int32_t threads,
                               int32_t* status_out, int32_t mem, void* stream) {
    if (!srv || (!jobs && n_jobs > 0)) return rid_fail(RID_ERR_ARG, "NULL argument");
    if (n_jobs < 0) return rid_fail(RID_ERR_ARG, "n_jobs=%d must be >= 0", n_jobs);
    if (threads != 0 && threads != 128 && threads != 256 && threads != 512)
        return rid_fail(RID_ERR_ARG, "threads=%d must be 0, 128, 256 or 512", threads);
    if (mem != RID_MEM_HOST && mem != RID_MEM_DEVICE) return rid_fail(RID_ERR_ARG, "mem must be RID_MEM_HOST or RID_MEM_DEVICE");
    if (n_jobs == 0) return RID_OK;
    STRY(check_server_device(srv));
    for (int k = 0; k < n_jobs; ++k) STRY(check_label_job(jobs[k], k, srv->device));
    cudaStream_t st = (cudaStream_t)stream;
    const bool host = mem == RID_MEM_HOST;

    // ---- device regions: one per job, plus the input / output staging
    std::vector<JobLayout> lay(n_jobs);
    std::vector<size_t> off(n_jobs, SIZE_MAX);
    size_t in_bytes = 0, out_bytes = 0;
    std::vector<size_t> in_off(n_jobs), out_off(n_jobs);
    int maxN = 0;
    size_t smem = 0;
    long long n_items = 0;
    for (int k = 0; k < n_jobs; ++k) {
        const rid_label_job& j = jobs[k];
        const SysDev* S = rid_sys_dev(j.sys);
        lay[k] = job_layout(j.n_runs, S->N, S->C, j.n_blocks);
        const size_t nb = (size_t)j.n_runs * S->N, nc = (size_t)j.n_runs * S->C;
        in_off[k] = in_bytes;
        in_bytes += align_up(12 * nb * (j.v0 ? 2 : 1) + 16 * nc);
        out_off[k] = out_bytes;
        out_bytes += align_up(24 * nc + 4 * (size_t)j.n_runs + 12 * nb * ((j.x_out ? 1 : 0) + (j.v_out ? 1 : 0)));
        maxN = std::max(maxN, S->N);
        smem = std::max(smem, rid_label_fused_smem(S->N, S->C, 0));
        n_items += j.n_runs;
    }
    if (n_items > (1 << 30)) return rid_fail(RID_ERR_ARG, "too many runs in one batch");
    size_t stage_in = SIZE_MAX, stage_out = SIZE_MAX;
    auto release = [&]() {
        for (int k = 0; k < n_jobs; ++k)
            if (off[k] != SIZE_MAX) srv->pool.free(off[k], lay[k].bytes);
        if (stage_in != SIZE_MAX) srv->pool.free(stage_in, in_bytes);
        if (stage_out != SIZE_MAX) srv->pool.free(stage_out, out_bytes);
    };
    for (int k = 0; k < n_jobs; ++k) {
        off[k] = srv->pool.alloc(lay[k].bytes);
        if (off[k] == SIZE_MAX) {
            release();
            return rid_fail(RID_ERR_OOM, "batch does not fit the server's HBM budget (%zu of %zu bytes in use)",
                            srv->pool.used(), srv->pool.capacity());
        }
    }
    if (host) {
        stage_in = srv->pool.alloc(in_bytes);
        stage_out = srv->pool.alloc(out_bytes);
        if (stage_in == SIZE_MAX || stage_out == SIZE_MAX) {
            release();
            return rid_fail(RID_ERR_OOM, "batch staging does not fit the server's HBM budget");
        }
    }
    char* pb = srv->pool.base();

    // ---- host-side tables
    std::vector<FusedJob> fj(n_jobs);
    std::vector<CopyDesc> din, dout;
    for (int k = 0; k < n_jobs; ++k) {
        const rid_label_job& j = jobs[k];
        const SysDev* S = rid_sys_dev(j.sys);
        const int R = j.n_runs, N = S->N, C = S->C;
        const size_t nb = (size_t)R * N, nc = (size_t)R * C;
        char* b = pb + off[k];
        const JobLayout& L = lay[k];
        FusedJob& J = fj[k];
        memset(&J, 0, sizeof(J));
        J.S = *S;
        J.x = reinterpret_cast<float4*>(b + L.x);
        J.v = reinterpret_cast<float4*>(b + L.v);
        J.f = reinterpret_cast<float4*>(b + L.f);
        J.s0 = reinterpret_cast<const double*>(b + L.s0);
        J.kappa = reinterpret_cast<const double*>(b + L.kappa);
        J.mf = reinterpret_cast<double*>(b + L.mf);
        J.se = reinterpret_cast<double*>(b + L.se);
        J.sd = reinterpret_cast<double*>(b + L.sd);
        J.sum = reinterpret_cast<double*>(b + L.sum);
        J.sum2 = reinterpret_cast<double*>(b + L.sum2);
        J.bsum = reinterpret_cast<double*>(b + L.bsum);
        J.flags = reinterpret_cast<int*>(b + L.flags);
        J.R = R;
        J.B = j.n_blocks;
        J.n_steps = j.n_steps;
        J.n_equil = j.n_equil;
        J.K = j.n_steps - j.n_equil;
        J.t0 = 0;
        J.t1 = j.n_steps;
        J.step0 = (uint32_t)j.step0;
        J.init = 1;
        J.mb = j.v0 ? 0 : 1;
        // inputs: caller arrays (device) or staging (host) -> pool
        const char* src = host ? pb + stage_in + in_off[k] : nullptr;
        size_t so = 0;
        auto in = [&](const void* user, size_t bytes) -> const void* {
            if (!host) return user;
            const void* at = src + so;
            so += bytes;
            return at;
        };
        din.push_back({in(j.x0, 12 * nb), J.x, (long long)nb, 0});
        if (j.v0) din.push_back({in(j.v0, 12 * nb), J.v, (long long)nb, 0});
        din.push_back({in(j.s0, 8 * nc), (void*)J.s0, (long long)nc, 2});
        din.push_back({in(j.kappa, 8 * nc), (void*)J.kappa, (long long)nc, 2});
        din.push_back({nullptr, b + L.sum, (long long)(L.zero_bytes / 4), 4});
        // outputs: pool -> caller arrays (device) or staging (host)
        char* dst = host ? pb + stage_out + out_off[k] : nullptr;
        size_t doff = 0;
        auto outp = [&](void* user, size_t bytes) -> void* {
            if (!host) return user;
            void* at = dst + doff;
            doff += bytes;
            return at;
        };
        dout.push_back({J.mf, outp(j.mf_out, 8 * nc), (long long)nc, 2});
        dout.push_back({J.se, outp(j.se_out, 8 * nc), (long long)nc, 2});
        dout.push_back({J.sd, outp(j.std_out, 8 * nc), (long long)nc, 2});
        dout.push_back({J.flags, host ? outp(nullptr, 4 * (size_t)R) : nullptr, (long long)R, 3});
        if (!host) dout.pop_back();   // flags are read separately below
        if (j.x_out) dout.push_back({J.x, outp(j.x_out, 12 * nb), (long long)nb, 1});
        if (j.v_out) dout.push_back({J.v, outp(j.v_out, 12 * nb), (long long)nb, 1});
    }
    // items, costliest first (all-pairs work grows as N^2 per step)
    std::vector<FusedItem> items;
    items.reserve((size_t)n_items);
    for (int k = 0; k < n_jobs; ++k)
        for (int r = 0; r < jobs[k].n_runs; ++r) items.push_back({k, r});
    std::stable_sort(items.begin(), items.end(), [&](const FusedItem& a, const FusedItem& b) {
        const double ca = (double)jobs[a.job].n_steps * fj[a.job].S.N * fj[a.job].S.N;
        const double cb = (double)jobs[b.job].n_steps * fj[b.job].S.N * fj[b.job].S.N;
        return ca > cb;
    });
    // flag copies for the device path go to a small pinned area instead
    std::vector<CopyDesc> dflags;
    if (!host)
        for (int k = 0; k < n_jobs; ++k) dflags.push_back({fj[k].flags, nullptr, (long long)fj[k].R, 3});

    // ---- metadata: [jobs | items | din | dout | counter], uploaded in one copy
    const size_t o_jobs = 0;
    const size_t o_items = align_up(o_jobs + sizeof(FusedJob) * n_jobs);
    const size_t o_din = align_up(o_items + sizeof(FusedItem) * items.size());
    const size_t o_dout = align_up(o_din + sizeof(CopyDesc) * din.size());
    const size_t o_cnt = align_up(o_dout + sizeof(CopyDesc) * (dout.size() + dflags.size()));
    const size_t o_flags = align_up(o_cnt + 16);
    size_t n_flag_words = 0;
    for (int k = 0; k < n_jobs; ++k) n_flag_words += (size_t)fj[k].R;
    const size_t meta_bytes = align_up(o_flags + 4 * n_flag_words);
    {
        const int rc = [&]() -> int {
            STRY(ensure_meta(srv, meta_bytes));
            STRY(srv->pin_meta.ensure(meta_bytes));
            if (host) {
                STRY(srv->pin_in.ensure(in_bytes));
                STRY(srv->pin_out.ensure(out_bytes));
            }
            return RID_OK;
        }();
        if (rc != RID_OK) {
            release();
            return rc;
        }
    }
    char* dm = static_cast<char*>(srv->d_meta);
    if (!host) {   // device path: flags land in the metadata area, then one copy to the host
        size_t fo = 0;
        for (auto& d : dflags) {
            d.dst = dm + o_flags + 4 * fo;
            fo += (size_t)d.n;
        }
    }
    char* hm = srv->pin_meta.c();
    memcpy(hm + o_jobs, fj.data(), sizeof(FusedJob) * n_jobs);
    memcpy(hm + o_items, items.data(), sizeof(FusedItem) * items.size());
    memcpy(hm + o_din, din.data(), sizeof(CopyDesc) * din.size());
    memcpy(hm + o_dout, dout.data(), sizeof(CopyDesc) * dout.size());
    if (!dflags.empty()) memcpy(hm + o_dout + sizeof(CopyDesc) * dout.size(), dflags.data(), sizeof(CopyDesc) * dflags.size());
    if (host) {
        for (int k = 0; k < n_jobs; ++k) {
            const rid_label_job& j = jobs[k];
            const SysDev* S = rid_sys_dev(j.sys);
            const size_t nb = (size_t)j.n_runs * S->N, nc = (size_t)j.n_runs * S->C;
            char* p = srv->pin_in.c() + in_off[k];
            memcpy(p, j.x0, 12 * nb);
            p += 12 * nb;
            if (j.v0) {
                memcpy(p, j.v0, 12 * nb);
                p += 12 * nb;
            }
            memcpy(p, j.s0, 8 * nc);
            p += 8 * nc;
            memcpy(p, j.kappa, 8 * nc);
        }
    }

    int rc = [&]() -> int {
        SCK(cudaMemcpyAsync(dm, hm, o_cnt, cudaMemcpyHostToDevice, st));
        if (host) SCK(cudaMemcpyAsync(pb + stage_in, srv->pin_in.p, in_bytes, cudaMemcpyHostToDevice, st));
        FusedArgs A{};
        A.jobs = reinterpret_cast<const FusedJob*>(dm + o_jobs);
        A.items = reinterpret_cast<const FusedItem*>(dm + o_items);
        A.n_items = (int)items.size();
        A.next = reinterpret_cast<int*>(dm + o_cnt);
        const CopyDesc* d_in = reinterpret_cast<const CopyDesc*>(dm + o_din);
        auto stage = [&]() -> int {
            rid_launch_copy_descs(d_in, (int)din.size(), st);
            SCK(cudaGetLastError());
            return RID_OK;
        };
        auto run = [&](int nt) -> int {
            const int occ = rid_label_fused_occupancy(nt, smem);
            if (occ < 1) return rid_fail(RID_ERR_CUDA, "k_label_fused<%d> cannot be resident with %zu bytes of shared memory", nt, smem);
            const int grid = (int)std::min<long long>(n_items, (long long)occ * srv->n_sm);
            SCK(cudaMemsetAsync(A.next, 0, sizeof(int), st));
            SCK(rid_launch_label_fused(A, nt, grid, smem, st));
            return RID_OK;
        };
        int nt = threads;
        const long long key = shape_key((int)n_items, maxN);
        if (nt == 0) {
            auto hit = srv->tuned.find(key);
            if (hit != srv->tuned.end()) nt = hit->second;
        }
        if (nt == 0) {
            // time a short prefix of the batch itself with each CTA size
            std::vector<FusedJob> trial = fj;
            long long tmin = 1ll << 60;
            for (const auto& J : trial) tmin = std::min(tmin, J.n_steps);
            const long long ts = std::min<long long>(8, tmin);
            for (auto& J : trial) J.t1 = ts;
            memcpy(hm + o_jobs, trial.data(), sizeof(FusedJob) * n_jobs);
            SCK(cudaMemcpyAsync(dm + o_jobs, hm + o_jobs, sizeof(FusedJob) * n_jobs, cudaMemcpyHostToDevice, st));
            cudaEvent_t e0, e1;
            SCK(cudaEventCreate(&e0));
            SCK(cudaEventCreate(&e1));
            float best = 1e30f;
            for (int cand : {128, 256, 512}) {
                if (rid_label_fused_occupancy(cand, smem) < 1) continue;
                STRY(stage());
                SCK(cudaEventRecord(e0, st));
                STRY(run(cand));
                SCK(cudaEventRecord(e1, st));
                SCK(cudaEventSynchronize(e1));
                float ms = 0.f;
                SCK(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) {
                    best = ms;
                    nt = cand;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (nt == 0) return rid_fail(RID_ERR_CUDA, "no CTA size of k_label_fused fits %zu bytes of shared memory", smem);
            srv->tuned[key] = nt;
            memcpy(hm + o_jobs, fj.data(), sizeof(FusedJob) * n_jobs);
            SCK(cudaMemcpyAsync(dm + o_jobs, hm + o_jobs, sizeof(FusedJob) * n_jobs, cudaMemcpyHostToDevice, st));
        }
        srv->last_threads = nt;
        STRY(stage());
        STRY(run(nt));
        rid_launch_copy_descs(reinterpret_cast<const CopyDesc*>(dm + o_dout), (int)(dout.size() + dflags.size()), st);
        SCK(cudaGetLastError());
        if (host) SCK(cudaMemcpyAsync(srv->pin_out.p, pb + stage_out, out_bytes, cudaMemcpyDeviceToHost, st));
        else SCK(cudaMemcpyAsync(hm + o_flags, dm + o_flags, 4 * n_flag_words, cudaMemcpyDeviceToHost, st));
        SCK(cudaStreamSynchronize(st));
        return RID_OK;
    }();
    if (rc != RID_OK) {
        cudaStreamSynchronize(st);
        release();
        return rc;
    }

    // ---- scatter host outputs, collect per-job status
    bool any_bad = false;
    size_t fo = 0;
    for (int k = 0; k < n_jobs; ++k) {
        const rid_label_job& j = jobs[k];
        const SysDev* S = rid_sys_dev(j.sys);
        const int R = j.n_runs;
        const size_t nb = (size_t)R * S->N, nc = (size_t)R * S->C;
        const int* fl;
        if (host) {
            const char* p = srv->pin_out.c() + out_off[k];
            memcpy(j.mf_out, p, 8 * nc);
            memcpy(j.se_out, p + 8 * nc, 8 * nc);
            memcpy(j.std_out, p + 16 * nc, 8 * nc);
            fl = reinterpret_cast<const int*>(p + 24 * nc);
            const char* q = p + 24 * nc + 4 * (size_t)R;
            if (j.x_out) {
                memcpy(j.x_out, q, 12 * nb);
                q += 12 * nb;
            }
            if (j.v_out) memcpy(j.v_out, q, 12 * nb);
        } else {
            fl = reinterpret_cast<const int*>(hm + o_flags) + fo;
            fo += (size_t)R;
        }
        bool bad = false;
        for (int r = 0; r < R; ++r) bad |= fl[r] != 0;
        if (status_out) status_out[k] = bad ? RID_ERR_NONFINITE : RID_OK;
        any_bad |= bad;
    }
    release();
    if (any_bad) return rid_fail(RID_ERR_NONFINITE, "non-finite force or velocity in at least one job");
    return RID_OK;
}
