// rid_server.cu -- the server object: device memory of a fixed budget
// (segments allocated on demand, first-fit inside each segment), pinned
// staging, batched restrained labeling through the persistent kernel
// k_label_fused (one launch for any number of uneven jobs) with a timing
// autotuner for its CTA size, and the request loop (rid_submit / rid_poll):
// a worker thread that admits jobs by device footprint and runs label jobs in
// ticks of the persistent kernel and exploration jobs as replayed CUDA graphs.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
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

// First-fit allocator over a range of offsets.  Free blocks are kept by
// offset and merged with their neighbours on release.
class OffsetAlloc {
  public:
    explicit OffsetAlloc(size_t bytes) { free_[0] = bytes; }
    size_t alloc(size_t n) {
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
    size_t used() const { return used_; }

  private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

// Device memory of the server: segments of at least seg_bytes, allocated on
// demand while the segments plus the reservations of exploration jobs (whose
// systems hold their own device memory) stay within the budget.  Empty
// segments are kept until trim() (cudaFree synchronises the device).
class SegPool {
  public:
    void init(size_t budget) {
        budget_ = budget;
        seg_bytes_ = std::min<size_t>(budget, (size_t)64 << 20);
    }
    // Device pointer to n bytes (256-byte aligned), or nullptr if it does not
    // fit the budget now (or cudaMalloc failed).
    void* alloc(size_t n) {
        n = align_up(n ? n : 1);
        for (auto& sg : segs_) {
            const size_t off = sg->a.alloc(n);
            if (off != SIZE_MAX) return sg->base + off;
        }
        const size_t sz = std::max(seg_bytes_, n);
        if (seg_total_ + reserved_ + sz > budget_) {
            trim();
            if (seg_total_ + reserved_ + sz > budget_) return nullptr;
        }
        void* p = nullptr;
        if (cudaMalloc(&p, sz) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        segs_.emplace_back(new Seg{static_cast<char*>(p), sz, OffsetAlloc(sz)});
        seg_total_ += sz;
        return segs_.back()->base + segs_.back()->a.alloc(n);
    }
    void free(void* p, size_t n) {
        if (!p) return;
        n = align_up(n ? n : 1);
        char* c = static_cast<char*>(p);
        for (auto& sg : segs_)
            if (c >= sg->base && c < sg->base + sg->bytes) {
                sg->a.free((size_t)(c - sg->base), n);
                return;
            }
    }
    bool reserve(size_t n) {
        if (seg_total_ + reserved_ + n > budget_) {
            trim();
            if (seg_total_ + reserved_ + n > budget_) return false;
        }
        reserved_ += n;
        return true;
    }
    void unreserve(size_t n) { reserved_ -= n; }
    void trim() {
        for (size_t i = 0; i < segs_.size();) {
            if (segs_[i]->a.used() == 0) {
                cudaFree(segs_[i]->base);
                seg_total_ -= segs_[i]->bytes;
                segs_.erase(segs_.begin() + i);
            } else {
                ++i;
            }
        }
    }
    void release() {
        for (auto& sg : segs_) cudaFree(sg->base);
        segs_.clear();
        seg_total_ = 0;
    }
    size_t budget() const { return budget_; }
    size_t in_use() const {
        size_t u = reserved_;
        for (auto& sg : segs_) u += sg->a.used();
        return u;
    }
    size_t held() const { return seg_total_ + reserved_; }

  private:
    struct Seg {
        char* base;
        size_t bytes;
        OffsetAlloc a;
    };
    std::vector<std::unique_ptr<Seg>> segs_;
    size_t budget_ = 0, seg_bytes_ = 0, seg_total_ = 0, reserved_ = 0;
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
namespace {

// One queued or running job of the request loop.
struct SJob {
    uint64_t id = 0;
    rid_request rq{};
    int W = 0, N = 0, C = 0, of = 1;
    long long T = 0;                     // exploration trace slots
    std::vector<float> x0, v0;
    std::vector<double> s0, kappa;
    size_t foot = 0;                     // bytes counted against the budget
    double t_submit = 0, t_start = -1, t_end = -1;
    int status = RID_NOT_READY;
    // label: one pool region = job arrays | input staging | output staging
    char* region = nullptr;
    JobLayout lay{};
    size_t in_off = 0, in_bytes = 0, out_off = 0, out_bytes = 0;
    FusedJob fj{};
    bool staged = false;
    long long t_done = 0, t_next = 0;
    // exploration
    int slot = -1, phase = 0;            // phase 1: chunk in flight, 2: final read in flight
    cudaGraphExec_t gexec = nullptr;
    long long chunk = 0, done = 0, cur = 0;
    char* dbuf = nullptr;                // pool: chunk traces, then final x / v
    size_t dbuf_bytes = 0;
};

struct ESlot {                           // stream of one running exploration job
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    Pinned pin;
    SJob* job = nullptr;
};

constexpr int N_ESLOTS = 16;

size_t label_io_in(const SJob& j) { return align_up(12 * (size_t)j.W * j.N * (j.v0.empty() ? 1 : 2) + 16 * (size_t)j.W * j.C); }
size_t label_io_out(const SJob& j) {
    return align_up(24 * (size_t)j.W * j.C + 4 * (size_t)j.W +
                    12 * (size_t)j.W * j.N * ((j.rq.x_out ? 1 : 0) + (j.rq.v_out ? 1 : 0)));
}
long long explore_chunk(int of, long long n_steps) {
    long long c = ((256 + of - 1) / of) * of;
    return std::max<long long>(of, std::min(c, (n_steps / of) * of));
}
size_t explore_dbuf(const SJob& j) {
    const size_t tc = (size_t)(explore_chunk(j.of, j.rq.n_steps) / j.of);
    return align_up(std::max((size_t)j.W * tc * (j.C + 1) * 4, (size_t)j.W * j.N * 24));
}

}  // namespace

struct rid_server {
    int device = 0, n_sm = 0;
    SegPool pool;
    std::mutex pool_mu;                  // pool and tuner cache: batch call and worker
    Pinned pin_in, pin_out, pin_meta;    // batch call staging
    void* d_meta = nullptr;              // batch call tables (grow-only, outside the budget)
    size_t d_meta_bytes = 0;
    std::map<long long, int> tuned;      // batch-shape key -> CTA size
    int last_threads = 0;
    // request loop
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;                       // queue, job records
    std::condition_variable cv;
    std::deque<SJob*> queue;
    std::unordered_map<uint64_t, std::unique_ptr<SJob>> jobs;
    uint64_t next_id = 1;
    int running = 0;
    bool stop = false;
    std::thread worker;
    // worker-owned
    cudaStream_t lst = nullptr;
    cudaEvent_t lev = nullptr, le0 = nullptr;
    // long chains' runs go to a second launch of thread-block clusters beside the tick's kernel
    cudaStream_t lst2 = nullptr;
    cudaEvent_t lfork = nullptr, ljoin = nullptr;
    std::vector<SJob*> labels;           // admitted label jobs
    std::vector<SJob*> tick;             // jobs of the tick in flight
    bool tick_busy = false;
    // per-step cost model of a label run, cost x (N + 200) ms, refined after every tick (measured
    // alone, one run per CTA: 9.2, 18.9 and 57.6 us per step at 200, 700 and 2000 beads, the
    // cluster-culled pairs growing about linearly in N)
    double tick_target_ms = 4.0, cost = 2.6e-5;
    double tick_pred = 0.0;
    Pinned lmeta_h, lio_h;
    void* lmeta_d = nullptr;
    size_t lmeta_d_bytes = 0;
    ESlot es[N_ESLOTS];
};

namespace {

double now_ms(const rid_server* srv) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - srv->t0).count();
}

int ensure_dev(void** p, size_t* have, size_t n) {
    if (n <= *have) return RID_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *have = 0;
    cudaError_t e = cudaMalloc(p, n);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return rid_fail(RID_ERR_OOM, "cudaMalloc(%zu) for server tables failed", n);
    }
    *have = n;
    return RID_OK;
}

int ensure_meta(rid_server* srv, size_t n) { return ensure_dev(&srv->d_meta, &srv->d_meta_bytes, n); }

int check_server_device(rid_server* srv) {
    int dev = -1;
    SCK(cudaGetDevice(&dev));
    if (dev != srv->device)
        return rid_fail(RID_ERR_STATE, "server was created on device %d, current device is %d", srv->device, dev);
    return RID_OK;
}

// The limits of rid_label plus the persistent kernel's shared-memory limit.
int check_label_args(rid_system* sys, int R, int B, uint64_t step0, int64_t n_steps, int64_t n_equil, int idx,
                     int device) {
    if (rid_sys_device(sys) != device)
        return rid_fail(RID_ERR_STATE, "job %d: system lives on device %d, server on %d", idx, rid_sys_device(sys),
                        device);
    if (R < 1) return rid_fail(RID_ERR_ARG, "job %d: n_runs=%d must be >= 1", idx, R);
    if (B < 2 || B > RID_MAX_BLOCKS) return rid_fail(RID_ERR_ARG, "job %d: n_blocks=%d outside [2, %d]", idx, B, RID_MAX_BLOCKS);
    if (n_equil < 0 || n_steps - n_equil < B)
        return rid_fail(RID_ERR_ARG, "job %d: need 0 <= n_equil and n_steps - n_equil >= n_blocks", idx);
    if (step0 + (uint64_t)n_steps > (1ull << 32)) return rid_fail(RID_ERR_ARG, "job %d: step0 + n_steps exceeds 2^32", idx);
    const SysDev* S = rid_sys_dev(sys);
    if (rid_label_fused_smem(S->N, S->C, 0) > LF_SMEM_LIMIT)
        return rid_fail(RID_ERR_ARG, "job %d: a chain of %d beads and %d CVs needs %zu bytes of shared memory (> %zu)",
                        idx, S->N, S->C, rid_label_fused_smem(S->N, S->C, 0), LF_SMEM_LIMIT);
    return RID_OK;
}

int check_label_job(const rid_label_job& j, int idx, int device) {
    if (!j.sys || !j.x0 || !j.s0 || !j.kappa || !j.mf_out || !j.se_out || !j.std_out)
        return rid_fail(RID_ERR_ARG, "job %d: NULL argument", idx);
    return check_label_args(j.sys, j.n_runs, j.n_blocks, j.step0, j.n_steps, j.n_equil, idx, device);
}

long long shape_key(int n_items, int maxN) {
    int a = 0, b = 0;
    while ((1 << a) < n_items && a < 30) ++a;
    while ((1 << b) < maxN && b < 30) ++b;
    return (long long)a * 64 + b;
}

// Fill the device pointers of a label job placed at `b`.
void place_label_job(FusedJob& J, char* b, const JobLayout& L, const SysDev& S, int R, int B, int64_t n_steps,
                     int64_t n_equil, uint64_t step0, bool mb) {
    memset(&J, 0, sizeof(J));
    J.S = S;
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
    J.B = B;
    J.n_steps = n_steps;
    J.n_equil = n_equil;
    J.K = n_steps - n_equil;
    J.t0 = 0;
    J.t1 = n_steps;
    J.step0 = (uint32_t)step0;
    J.init = 1;
    J.mb = mb ? 1 : 0;
}

// Descriptors that move a label job's inputs (from staging or from caller
// device arrays) into its arrays and zero its accumulators.
void label_in_descs(std::vector<CopyDesc>& d, const FusedJob& J, const JobLayout& L, char* region, const void* x0,
                    const void* v0, const void* s0, const void* kappa) {
    const long long nb = (long long)J.R * J.S.N, nc = (long long)J.R * J.S.C;
    d.push_back({x0, J.x, nb, 0});
    if (v0) d.push_back({v0, J.v, nb, 0});
    d.push_back({s0, (void*)J.s0, nc, 2});
    d.push_back({kappa, (void*)J.kappa, nc, 2});
    d.push_back({nullptr, region + L.sum, (long long)(L.zero_bytes / 4), 4});
}

// Descriptors that move a label job's results into `dst` laid out as
// mf | se | sd | flags | x? | v?.
void label_out_descs(std::vector<CopyDesc>& d, const FusedJob& J, char* dst, bool xo, bool vo) {
    const long long nb = (long long)J.R * J.S.N, nc = (long long)J.R * J.S.C;
    d.push_back({J.mf, dst, nc, 2});
    d.push_back({J.se, dst + 8 * nc, nc, 2});
    d.push_back({J.sd, dst + 16 * nc, nc, 2});
    d.push_back({J.flags, dst + 24 * nc, J.R, 3});
    char* q = dst + 24 * nc + 4 * J.R;
    if (xo) {
        d.push_back({J.x, q, nb, 1});
        q += 12 * nb;
    }
    if (vo) d.push_back({J.v, q, nb, 1});
}

}  // namespace

// ---------------------------------------------------------------------------
// The request loop.
namespace {

void finish_job(rid_server* srv, SJob* j, int status) {
    std::lock_guard<std::mutex> lk(srv->mu);
    j->status = status;
    j->t_end = now_ms(srv);
    --srv->running;
    srv->cv.notify_all();
}

// Admission of a queued job: 0 admitted, 1 no device memory within the budget
// now, 2 waiting for a stream slot or for its system to become idle.
int try_admit(rid_server* srv, SJob* j) {
    std::lock_guard<std::mutex> lk(srv->pool_mu);
    if (j->rq.kind == RID_JOB_LABEL) {
        void* p = srv->pool.alloc(j->foot);
        if (!p) return 1;
        j->region = static_cast<char*>(p);
        return 0;
    }
    int slot = -1;
    for (int k = 0; k < N_ESLOTS; ++k) {
        if (srv->es[k].job && srv->es[k].job->rq.sys == j->rq.sys) return 2;   // system busy
        if (!srv->es[k].job && slot < 0) slot = k;
    }
    if (slot < 0) return 2;
    const size_t sys_bytes = j->foot - j->dbuf_bytes;
    if (!srv->pool.reserve(sys_bytes)) return 1;
    void* p = srv->pool.alloc(j->dbuf_bytes);
    if (!p) {
        srv->pool.unreserve(sys_bytes);
        return 1;
    }
    j->dbuf = static_cast<char*>(p);
    j->slot = slot;
    srv->es[slot].job = j;
    return 0;
}

void release_job_memory(rid_server* srv, SJob* j) {
    std::lock_guard<std::mutex> lk(srv->pool_mu);
    if (j->rq.kind == RID_JOB_LABEL) {
        srv->pool.free(j->region, j->foot);
        j->region = nullptr;
    } else {
        srv->pool.free(j->dbuf, j->dbuf_bytes);
        srv->pool.unreserve(j->foot - j->dbuf_bytes);
        j->dbuf = nullptr;
        srv->es[j->slot].job = nullptr;
        rid_sys_serving(j->rq.sys, false);
    }
}

// ---- exploration jobs
int explore_launch_chunk(rid_server* srv, SJob* j) {
    NvtxScope nvtx_("explore chunk");
    ESlot& e = srv->es[j->slot];
    rid_system* sys = j->rq.sys;
    j->cur = std::min(j->chunk, j->rq.n_steps - j->done);
    float* dcv = reinterpret_cast<float*>(j->dbuf);
    const long long tc = j->cur / j->of;
    float* deps = dcv + (size_t)j->W * tc * j->C;
    if (j->gexec && j->cur == j->chunk) {
        SCK(cudaGraphLaunch(j->gexec, e.st));
    } else {
        STRY(rid_sys_advance(sys, j->cur, dcv, deps, e.st));
    }
    if (tc > 0 && (j->rq.cv_out || j->rq.eps_out)) {
        const size_t bytes = (size_t)j->W * tc * (j->C + 1) * 4;
        STRY(e.pin.ensure(bytes));
        SCK(cudaMemcpyAsync(e.pin.p, j->dbuf, bytes, cudaMemcpyDeviceToHost, e.st));
    }
    SCK(cudaEventRecord(e.ev, e.st));
    j->phase = 1;
    return RID_OK;
}

int explore_start(rid_server* srv, SJob* j) {
    ESlot& e = srv->es[j->slot];
    rid_system* sys = j->rq.sys;
    rid_sys_serving(sys, true);
    STRY(rid_sys_load(sys, j->W, j->x0.data(), j->v0.empty() ? nullptr : j->v0.data(), j->rq.step0, e.st));
    j->chunk = explore_chunk(j->of, j->rq.n_steps);
    if (j->rq.n_steps >= j->chunk) {
        float* dcv = reinterpret_cast<float*>(j->dbuf);
        float* deps = dcv + (size_t)j->W * (j->chunk / j->of) * j->C;
        STRY(rid_sys_graph_advance(sys, j->chunk, dcv, deps, e.st, &j->gexec));
    }
    return explore_launch_chunk(srv, j);
}

// Returns true when the job made progress.
bool explore_progress(rid_server* srv, SJob* j) {
    ESlot& e = srv->es[j->slot];
    const cudaError_t q = cudaEventQuery(e.ev);
    if (q == cudaErrorNotReady) return false;
    int rc = RID_OK;
    if (q != cudaSuccess) rc = rid_fail(RID_ERR_CUDA, "exploration job: %s", cudaGetErrorString(q));
    if (rc == RID_OK && j->phase == 1) {
        const long long tc = j->cur / j->of, s0 = j->done / j->of;
        const float* pc = static_cast<const float*>(e.pin.p);
        const float* pe = pc + (size_t)j->W * tc * j->C;
        for (int w = 0; w < j->W && tc > 0; ++w) {
            if (j->rq.cv_out)
                memcpy(j->rq.cv_out + ((size_t)w * j->T + s0) * j->C, pc + (size_t)w * tc * j->C, 4 * tc * j->C);
            if (j->rq.eps_out) memcpy(j->rq.eps_out + (size_t)w * j->T + s0, pe + (size_t)w * tc, 4 * tc);
        }
        j->done += j->cur;
        if (j->done < j->rq.n_steps) {
            rc = explore_launch_chunk(srv, j);
            if (rc == RID_OK) return true;
        } else {
            float* dx = reinterpret_cast<float*>(j->dbuf);
            float* dv = dx + (size_t)j->W * j->N * 3;
            rc = rid_sys_read_async(j->rq.sys, dx, dv, e.st);
            if (rc == RID_OK) rc = e.pin.ensure((size_t)j->W * j->N * 24);
            if (rc == RID_OK && cudaMemcpyAsync(e.pin.p, j->dbuf, (size_t)j->W * j->N * 24, cudaMemcpyDeviceToHost,
                                                e.st) != cudaSuccess)
                rc = rid_fail(RID_ERR_CUDA, "exploration job: copy of the final state failed");
            if (rc == RID_OK && cudaEventRecord(e.ev, e.st) != cudaSuccess) rc = rid_fail(RID_ERR_CUDA, "event record");
            if (rc == RID_OK) {
                j->phase = 2;
                return true;
            }
        }
    } else if (rc == RID_OK && j->phase == 2) {
        const size_t nb3 = (size_t)j->W * j->N * 3;
        const float* p = static_cast<const float*>(e.pin.p);
        if (j->rq.x_out) memcpy(j->rq.x_out, p, 4 * nb3);
        if (j->rq.v_out) memcpy(j->rq.v_out, p + nb3, 4 * nb3);
        bool bad = false;
        rc = rid_sys_flags(j->rq.sys, e.st, &bad);
        if (rc == RID_OK && bad) rc = RID_ERR_NONFINITE;
    }
    // final (done, or failed)
    cudaStreamSynchronize(e.st);
    if (j->gexec) cudaGraphExecDestroy(j->gexec);
    j->gexec = nullptr;
    release_job_memory(srv, j);
    finish_job(srv, j, rc);
    return true;
}

// Label runs of chains of at least LF_CL_MIN_N beads go to a second launch of
// the persistent kernel in thread-block clusters of LF_CL CTAs, beside the
// tick's main launch; the cost model counts their steps as LF_CL_SPEED times
// cheaper.
constexpr int LF_CL_MIN_N = 768;
constexpr int LF_CL = 4;
constexpr double LF_CL_SPEED = 2.5;

// ---- label jobs: one tick of the persistent kernel over every admitted job
int label_tick_launch(rid_server* srv) {
    NvtxScope nvtx_("label tick");
    std::vector<SJob*> act;
    for (SJob* j : srv->labels) act.push_back(j);
    if (act.empty()) return RID_OK;
    cudaStream_t st = srv->lst;
    // steps per job: about tick_target_ms of work for the job's chain length
    std::vector<FusedJob> fj(act.size());
    std::vector<CopyDesc> din, dout;
    std::vector<FusedItem> items;
    size_t in_h = 0, out_h = 0;
    double pred = 0.0;
    int maxN = 0;
    size_t smem = 0, smem_cl = 0;
    for (size_t k = 0; k < act.size(); ++k) {
        SJob* j = act[k];
        const bool cl = j->N >= LF_CL_MIN_N;
        const double per = srv->cost * ((double)j->N / (cl ? LF_CL_SPEED : 1.0) + 200.0);
        long long steps = (long long)(srv->tick_target_ms / per);
        steps = std::max<long long>(8, steps);
        steps = std::min<long long>(steps, j->rq.n_steps - j->t_done);
        FusedJob J = j->fj;
        J.t0 = j->t_done;
        J.t1 = j->t_done + steps;
        J.init = j->t_done == 0 ? 1 : 0;
        j->t_next = J.t1;
        fj[k] = J;
        pred = std::max(pred, per * steps);
        maxN = std::max(maxN, j->N);
        (cl ? smem_cl : smem) = std::max(cl ? smem_cl : smem, rid_label_fused_smem(j->N, j->C, 0));
        for (int r = 0; r < j->W; ++r) items.push_back({(int)k, r});
        if (!j->staged) {
            // staging order s0 | kappa | x0 | v0: the doubles first, so every array stays aligned
            char* src = j->region + j->in_off;
            const size_t nb = (size_t)j->W * j->N, nc = (size_t)j->W * j->C;
            const char* x0 = src + 16 * nc;
            const char* v0 = j->v0.empty() ? nullptr : x0 + 12 * nb;
            label_in_descs(din, J, j->lay, j->region, x0, v0, src, src + 8 * nc);
            in_h += j->in_bytes;
        }
        if (J.t1 == j->rq.n_steps) {
            label_out_descs(dout, J, j->region + j->out_off, j->rq.x_out != nullptr, j->rq.v_out != nullptr);
            out_h += j->out_bytes;
        }
    }
    std::stable_sort(items.begin(), items.end(), [&](const FusedItem& a, const FusedItem& b) {
        return (fj[a.job].t1 - fj[a.job].t0) * (double)fj[a.job].S.N * fj[a.job].S.N >
               (fj[b.job].t1 - fj[b.job].t0) * (double)fj[b.job].S.N * fj[b.job].S.N;
    });
    // the short chains' items first (the main launch), then the long chains' (the clusters)
    std::stable_partition(items.begin(), items.end(),
                          [&](const FusedItem& a) { return fj[a.job].S.N < LF_CL_MIN_N; });
    int n_small = 0;
    while (n_small < (int)items.size() && fj[items[n_small].job].S.N < LF_CL_MIN_N) ++n_small;
    const int n_big = (int)items.size() - n_small;
    // host staging of new inputs, then the tables
    STRY(srv->lio_h.ensure(std::max(in_h, out_h) + 256));
    const size_t o_items = align_up(sizeof(FusedJob) * fj.size());
    const size_t o_din = align_up(o_items + sizeof(FusedItem) * items.size());
    const size_t o_dout = align_up(o_din + sizeof(CopyDesc) * din.size());
    const size_t o_cnt = align_up(o_dout + sizeof(CopyDesc) * dout.size());
    const size_t meta = o_cnt + 256;
    STRY(srv->lmeta_h.ensure(meta));
    STRY(ensure_dev(&srv->lmeta_d, &srv->lmeta_d_bytes, meta));
    char* hm = srv->lmeta_h.c();
    char* dm = static_cast<char*>(srv->lmeta_d);
    memcpy(hm, fj.data(), sizeof(FusedJob) * fj.size());
    memcpy(hm + o_items, items.data(), sizeof(FusedItem) * items.size());
    if (!din.empty()) memcpy(hm + o_din, din.data(), sizeof(CopyDesc) * din.size());
    if (!dout.empty()) memcpy(hm + o_dout, dout.data(), sizeof(CopyDesc) * dout.size());
    SCK(cudaMemcpyAsync(dm, hm, o_cnt, cudaMemcpyHostToDevice, st));
    size_t ho = 0;
    for (SJob* j : act) {
        if (j->staged) continue;
        char* p = srv->lio_h.c() + ho;
        const size_t nb = (size_t)j->W * j->N, nc = (size_t)j->W * j->C;
        size_t o = 0;
        memcpy(p + o, j->s0.data(), 8 * nc);
        o += 8 * nc;
        memcpy(p + o, j->kappa.data(), 8 * nc);
        o += 8 * nc;
        memcpy(p + o, j->x0.data(), 12 * nb);
        o += 12 * nb;
        if (!j->v0.empty()) memcpy(p + o, j->v0.data(), 12 * nb);
        SCK(cudaMemcpyAsync(j->region + j->in_off, p, j->in_bytes, cudaMemcpyHostToDevice, st));
        ho += j->in_bytes;
        j->staged = true;
    }
    if (!din.empty()) rid_launch_copy_descs(reinterpret_cast<const CopyDesc*>(dm + o_din), (int)din.size(), st);
    FusedArgs A{};
    A.jobs = reinterpret_cast<const FusedJob*>(dm);
    A.items = reinterpret_cast<const FusedItem*>(dm + o_items);
    A.n_items = n_small;
    A.next = reinterpret_cast<int*>(dm + o_cnt);
    FusedArgs A2 = A;
    A2.items = A.items + n_small;
    A2.n_items = n_big;
    A2.next = reinterpret_cast<int*>(dm + o_cnt + 128);
    int nt = 256;
    {
        std::lock_guard<std::mutex> lk(srv->pool_mu);
        auto hit = srv->tuned.find(shape_key((int)items.size(), maxN));
        if (hit != srv->tuned.end()) nt = hit->second;
    }
    const size_t smem_all = std::max(smem, smem_cl);
    if (rid_label_fused_occupancy(nt, smem_all) < 1) nt = 128;
    SCK(cudaMemsetAsync(A.next, 0, 256, st));
    SCK(cudaEventRecord(srv->le0, st));
    if (n_big > 0) {
        const int occ_cl = std::max(1, rid_label_fused_occupancy(nt, smem_cl));
        const long long clusters = std::max<long long>(1, (long long)occ_cl * srv->n_sm / LF_CL);
        const int grid_cl = (int)(std::min<long long>(n_big, clusters) * LF_CL);
        SCK(cudaEventRecord(srv->lfork, st));
        SCK(cudaStreamWaitEvent(srv->lst2, srv->lfork, 0));
        if (rid_launch_label_fused(A2, nt, grid_cl, smem_cl, srv->lst2, LF_CL) != cudaSuccess) {
            // a cluster launch the device refuses: the same items one CTA per run (the same bits)
            (void)cudaGetLastError();
            const int grid1 = (int)std::min<long long>(n_big, (long long)occ_cl * srv->n_sm);
            SCK(rid_launch_label_fused(A2, nt, grid1, smem_cl, srv->lst2, 1));
        }
        SCK(cudaEventRecord(srv->ljoin, srv->lst2));
    }
    if (n_small > 0) {
        const int occ = std::max(1, rid_label_fused_occupancy(nt, smem));
        const int grid = (int)std::min<long long>(n_small, (long long)occ * srv->n_sm);
        SCK(rid_launch_label_fused(A, nt, grid, smem, st));
    }
    if (n_big > 0) SCK(cudaStreamWaitEvent(st, srv->ljoin, 0));
    if (!dout.empty()) rid_launch_copy_descs(reinterpret_cast<const CopyDesc*>(dm + o_dout), (int)dout.size(), st);
    SCK(cudaEventRecord(srv->lev, st));
    ho = 0;
    for (size_t k = 0; k < act.size(); ++k) {
        SJob* j = act[k];
        if (j->t_next != j->rq.n_steps) continue;
        SCK(cudaMemcpyAsync(srv->lio_h.c() + ho, j->region + j->out_off, j->out_bytes, cudaMemcpyDeviceToHost, st));
        ho += j->out_bytes;
    }
    SCK(cudaEventRecord(srv->lev, st));
    srv->tick = act;
    srv->tick_pred = pred;
    srv->tick_busy = true;
    return RID_OK;
}

bool label_tick_progress(rid_server* srv) {
    if (!srv->tick_busy) return false;
    const cudaError_t q = cudaEventQuery(srv->lev);
    if (q == cudaErrorNotReady) return false;
    srv->tick_busy = false;
    int rc = q == cudaSuccess ? RID_OK : rid_fail(RID_ERR_CUDA, "label tick: %s", cudaGetErrorString(q));
    // refine the cost model from the kernel's time (its longest item sets it)
    float ms = 0.f;
    if (rc == RID_OK && cudaEventElapsedTime(&ms, srv->le0, srv->lev) == cudaSuccess && srv->tick_pred > 0.0) {
        const double ratio = ms / srv->tick_pred;
        srv->cost *= std::min(4.0, std::max(0.25, 0.5 + 0.5 * ratio));
    }
    size_t ho = 0;
    std::vector<SJob*> keep;
    for (SJob* j : srv->labels) {
        if (rc != RID_OK) {
            release_job_memory(srv, j);
            finish_job(srv, j, rc);
            continue;
        }
        j->t_done = j->t_next;
        if (j->t_done < j->rq.n_steps) {
            keep.push_back(j);
            continue;
        }
        const char* p = srv->lio_h.c() + ho;
        ho += j->out_bytes;
        const size_t nb = (size_t)j->W * j->N, nc = (size_t)j->W * j->C;
        memcpy(j->rq.mf_out, p, 8 * nc);
        memcpy(j->rq.se_out, p + 8 * nc, 8 * nc);
        memcpy(j->rq.std_out, p + 16 * nc, 8 * nc);
        const int* fl = reinterpret_cast<const int*>(p + 24 * nc);
        bool bad = false;
        for (int r = 0; r < j->W; ++r) bad |= fl[r] != 0;
        const char* q2 = p + 24 * nc + 4 * (size_t)j->W;
        if (j->rq.x_out) {
            memcpy(j->rq.x_out, q2, 12 * nb);
            q2 += 12 * nb;
        }
        if (j->rq.v_out) memcpy(j->rq.v_out, q2, 12 * nb);
        release_job_memory(srv, j);
        finish_job(srv, j, bad ? RID_ERR_NONFINITE : RID_OK);
    }
    srv->labels.swap(keep);
    srv->tick.clear();
    return true;
}

void worker_main(rid_server* srv) {
    cudaSetDevice(srv->device);
    for (;;) {
        std::vector<SJob*> admitted;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            for (;;) {
                const bool busy = srv->running > 0;
                if (srv->stop && srv->queue.empty() && !busy) return;
                if (!srv->queue.empty() || busy) break;
                srv->cv.wait(lk);
            }
            // arrival order; a job short of memory stops admission (so large jobs
            // are not starved), one waiting for a slot or its system is passed over
            for (auto it = srv->queue.begin(); it != srv->queue.end();) {
                SJob* j = *it;
                const int a = try_admit(srv, j);
                if (a == 1) break;
                if (a == 2) {
                    ++it;
                    continue;
                }
                it = srv->queue.erase(it);
                ++srv->running;
                j->t_start = now_ms(srv);
                admitted.push_back(j);
            }
        }
        bool moved = !admitted.empty();
        for (SJob* j : admitted) {
            if (j->rq.kind == RID_JOB_LABEL) {
                place_label_job(j->fj, j->region, j->lay, *rid_sys_dev(j->rq.sys), j->W, j->rq.n_blocks,
                                j->rq.n_steps, j->rq.n_equil, j->rq.step0, j->v0.empty());
                srv->labels.push_back(j);
            } else {
                const int rc = explore_start(srv, j);
                if (rc != RID_OK) {
                    cudaStreamSynchronize(srv->es[j->slot].st);
                    if (j->gexec) cudaGraphExecDestroy(j->gexec);
                    j->gexec = nullptr;
                    release_job_memory(srv, j);
                    finish_job(srv, j, rc);
                }
            }
        }
        moved |= label_tick_progress(srv);
        if (!srv->tick_busy && !srv->labels.empty()) {
            const int rc = label_tick_launch(srv);
            if (rc != RID_OK) {
                cudaStreamSynchronize(srv->lst);
                for (SJob* j : srv->labels) {
                    release_job_memory(srv, j);
                    finish_job(srv, j, rc);
                }
                srv->labels.clear();
            }
            moved = true;
        }
        for (int k = 0; k < N_ESLOTS; ++k)
            if (srv->es[k].job) moved |= explore_progress(srv, srv->es[k].job);
        if (!moved) {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv.wait_for(lk, std::chrono::microseconds(100));
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" int rid_server_create(uint64_t budget, rid_server** out) {
    if (!out) return rid_fail(RID_ERR_ARG, "NULL out");
    *out = nullptr;
    if (budget < (1u << 20)) return rid_fail(RID_ERR_ARG, "hbm_budget_bytes=%llu below 1 MiB", (unsigned long long)budget);
    std::unique_ptr<rid_server> srv(new rid_server());
    srv->t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaGetDevice(&srv->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&srv->n_sm, cudaDevAttrMultiProcessorCount, srv->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&srv->lst, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&srv->lev);
    if (e == cudaSuccess) e = cudaEventCreate(&srv->le0);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&srv->lst2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&srv->lfork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&srv->ljoin, cudaEventDisableTiming);
    for (int k = 0; k < N_ESLOTS && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&srv->es[k].st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&srv->es[k].ev, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return rid_fail(RID_ERR_CUDA, "rid_server_create: %s", cudaGetErrorString(e));
    srv->pool.init((size_t)budget);
    rid_server* p = srv.release();
    p->worker = std::thread(worker_main, p);
    *out = p;
    return RID_OK;
}

extern "C" int rid_server_destroy(rid_server* srv) {
    if (!srv) return RID_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    cudaDeviceSynchronize();
    srv->pool.release();
    srv->pin_in.release();
    srv->pin_out.release();
    srv->pin_meta.release();
    srv->lmeta_h.release();
    srv->lio_h.release();
    if (srv->d_meta) cudaFree(srv->d_meta);
    if (srv->lmeta_d) cudaFree(srv->lmeta_d);
    for (int k = 0; k < N_ESLOTS; ++k) {
        srv->es[k].pin.release();
        if (srv->es[k].ev) cudaEventDestroy(srv->es[k].ev);
        if (srv->es[k].st) cudaStreamDestroy(srv->es[k].st);
    }
    if (srv->lev) cudaEventDestroy(srv->lev);
    if (srv->le0) cudaEventDestroy(srv->le0);
    if (srv->lst) cudaStreamDestroy(srv->lst);
    if (srv->lfork) cudaEventDestroy(srv->lfork);
    if (srv->ljoin) cudaEventDestroy(srv->ljoin);
    if (srv->lst2) cudaStreamDestroy(srv->lst2);
    delete srv;
    return RID_OK;
}

extern "C" int rid_submit(rid_server* srv, const rid_request* req, uint64_t* job_id) {
    if (!srv || !req || !job_id) return rid_fail(RID_ERR_ARG, "NULL argument");
    const rid_request& q = *req;
    if (q.kind != RID_JOB_LABEL && q.kind != RID_JOB_EXPLORE) return rid_fail(RID_ERR_ARG, "kind=%d is not a job kind", q.kind);
    if (!q.sys || !q.x0) return rid_fail(RID_ERR_ARG, "NULL sys or x0");
    if (q.n_walkers < 1) return rid_fail(RID_ERR_ARG, "n_walkers=%d must be >= 1", q.n_walkers);
    if (q.n_steps < 1) return rid_fail(RID_ERR_ARG, "n_steps must be >= 1");
    const SysDev* S = rid_sys_dev(q.sys);
    std::unique_ptr<SJob> j(new SJob());
    j->rq = q;
    j->W = q.n_walkers;
    j->N = S->N;
    j->C = S->C;
    j->of = S->output_freq > 0 ? S->output_freq : 1;
    const size_t nb = (size_t)j->W * j->N, nc = (size_t)j->W * j->C;
    if (q.kind == RID_JOB_LABEL) {
        if (!q.s0 || !q.kappa || !q.mf_out || !q.se_out || !q.std_out) return rid_fail(RID_ERR_ARG, "label job: NULL argument");
        STRY(check_label_args(q.sys, q.n_walkers, q.n_blocks, q.step0, q.n_steps, q.n_equil, 0, srv->device));
    } else {
        if (rid_sys_device(q.sys) != srv->device) return rid_fail(RID_ERR_STATE, "system lives on another device");
        if (q.step0 + (uint64_t)q.n_steps > (1ull << 32)) return rid_fail(RID_ERR_ARG, "step0 + n_steps exceeds 2^32");
        j->T = q.n_steps / j->of;
    }
    j->x0.assign(q.x0, q.x0 + 3 * nb);
    if (q.v0) j->v0.assign(q.v0, q.v0 + 3 * nb);
    if (q.kind == RID_JOB_LABEL) {
        j->s0.assign(q.s0, q.s0 + nc);
        j->kappa.assign(q.kappa, q.kappa + nc);
        j->lay = job_layout(j->W, j->N, j->C, q.n_blocks);
        j->in_off = j->lay.bytes;
        j->in_bytes = label_io_in(*j);
        j->out_off = j->in_off + j->in_bytes;
        j->out_bytes = label_io_out(*j);
        j->foot = j->out_off + j->out_bytes;
    } else {
        j->dbuf_bytes = explore_dbuf(*j);
        j->foot = rid_sys_footprint(q.sys, j->W) + j->dbuf_bytes;
    }
    if (j->foot > srv->pool.budget())
        return rid_fail(RID_ERR_OOM, "job needs %zu bytes, more than the server's budget of %zu", j->foot,
                        srv->pool.budget());
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) return rid_fail(RID_ERR_STATE, "server is shutting down");
    j->id = srv->next_id++;
    j->t_submit = now_ms(srv);
    *job_id = j->id;
    SJob* raw = j.get();
    srv->jobs[j->id] = std::move(j);
    srv->queue.push_back(raw);
    srv->cv.notify_all();
    return RID_OK;
}

extern "C" int rid_poll(rid_server* srv, uint64_t job_id, rid_job_info* info) {
    if (!srv) return rid_fail(RID_ERR_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end()) return rid_fail(RID_ERR_ARG, "unknown job id %llu", (unsigned long long)job_id);
    SJob* j = it->second.get();
    if (info) {
        info->status = j->status;
        info->kind = j->rq.kind;
        info->t_submit_ms = j->t_submit;
        info->t_start_ms = j->t_start;
        info->t_end_ms = j->t_end;
    }
    const int st = j->status;
    if (st == RID_NOT_READY) return RID_NOT_READY;
    // rid_fail keeps a message for this thread only for the failing statuses
    if (st != RID_OK) rid_fail(st, "job %llu finished with status %d", (unsigned long long)job_id, st);
    srv->jobs.erase(it);
    return st;
}

extern "C" int rid_cancel(rid_server* srv, uint64_t job_id) {
    if (!srv) return rid_fail(RID_ERR_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end()) return rid_fail(RID_ERR_ARG, "unknown job id %llu", (unsigned long long)job_id);
    SJob* j = it->second.get();
    // only a job still waiting for admission holds nothing on the device; the
    // worker reads the queue under the same lock
    auto q = std::find(srv->queue.begin(), srv->queue.end(), j);
    if (q == srv->queue.end())
        return rid_fail(RID_ERR_STATE, "job %llu is %s", (unsigned long long)job_id,
                        j->status == RID_NOT_READY ? "running" : "final");
    srv->queue.erase(q);
    j->status = RID_ERR_CANCELLED;
    j->t_end = now_ms(srv);
    srv->cv.notify_all();
    return RID_OK;
}

extern "C" int rid_server_load(rid_server* srv, int32_t* queued, int32_t* running, uint64_t* bytes_in_use) {
    if (!srv) return rid_fail(RID_ERR_ARG, "NULL server");
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (queued) *queued = (int32_t)srv->queue.size();
        if (running) *running = srv->running;
    }
    std::lock_guard<std::mutex> lk(srv->pool_mu);
    if (bytes_in_use) *bytes_in_use = srv->pool.in_use();
    return RID_OK;
}

extern "C" int rid_label_batch(rid_server* srv, const rid_label_job* jobs, int32_t n_jobs, int32_t threads,
                               int32_t* status_out, int32_t mem, void* stream) {
    NvtxScope nvtx_("rid_label_batch");
    if (!srv || (!jobs && n_jobs > 0)) return rid_fail(RID_ERR_ARG, "NULL argument");
    if (n_jobs < 0) return rid_fail(RID_ERR_ARG, "n_jobs=%d must be >= 0", n_jobs);
    if (threads != 0 && threads != 128 && threads != 256 && threads != 512)
        return rid_fail(RID_ERR_ARG, "threads=%d must be 0, 128, 256 or 512", threads);
    if (mem != RID_MEM_HOST && mem != RID_MEM_DEVICE) return rid_fail(RID_ERR_ARG, "mem must be RID_MEM_HOST or RID_MEM_DEVICE");
    if (n_jobs == 0) return RID_OK;
    STRY(check_server_device(srv));
    for (int k = 0; k < n_jobs; ++k) STRY(check_label_job(jobs[k], k, srv->device));
    std::lock_guard<std::mutex> pool_lock(srv->pool_mu);
    cudaStream_t st = (cudaStream_t)stream;
    const bool host = mem == RID_MEM_HOST;

    // ---- device regions: one per job, plus the input / output staging
    std::vector<JobLayout> lay(n_jobs);
    std::vector<char*> off(n_jobs, nullptr);
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
    char* stage_in = nullptr;
    char* stage_out = nullptr;
    auto release = [&]() {
        for (int k = 0; k < n_jobs; ++k)
            if (off[k]) srv->pool.free(off[k], lay[k].bytes);
        if (stage_in) srv->pool.free(stage_in, in_bytes);
        if (stage_out) srv->pool.free(stage_out, out_bytes);
    };
    for (int k = 0; k < n_jobs; ++k) {
        off[k] = static_cast<char*>(srv->pool.alloc(lay[k].bytes));
        if (!off[k]) {
            release();
            return rid_fail(RID_ERR_OOM, "batch does not fit the server's HBM budget (%zu of %zu bytes in use)",
                            srv->pool.in_use(), srv->pool.budget());
        }
    }
    if (host) {
        stage_in = static_cast<char*>(srv->pool.alloc(in_bytes));
        stage_out = static_cast<char*>(srv->pool.alloc(out_bytes));
        if (!stage_in || !stage_out) {
            release();
            return rid_fail(RID_ERR_OOM, "batch staging does not fit the server's HBM budget");
        }
    }

    // ---- host-side tables
    std::vector<FusedJob> fj(n_jobs);
    std::vector<CopyDesc> din, dout;
    for (int k = 0; k < n_jobs; ++k) {
        const rid_label_job& j = jobs[k];
        const SysDev* S = rid_sys_dev(j.sys);
        const int R = j.n_runs, N = S->N, C = S->C;
        const size_t nb = (size_t)R * N, nc = (size_t)R * C;
        char* b = off[k];
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
        const char* src = host ? stage_in + in_off[k] : nullptr;
        size_t so = 0;
        auto in = [&](const void* user, size_t bytes) -> const void* {
            if (!host) return user;
            const void* at = src + so;
            so += bytes;
            return at;
        };
        // staging order: the doubles first, so every array stays aligned
        din.push_back({in(j.s0, 8 * nc), (void*)J.s0, (long long)nc, 2});
        din.push_back({in(j.kappa, 8 * nc), (void*)J.kappa, (long long)nc, 2});
        din.push_back({in(j.x0, 12 * nb), J.x, (long long)nb, 0});
        if (j.v0) din.push_back({in(j.v0, 12 * nb), J.v, (long long)nb, 0});
        din.push_back({nullptr, b + L.sum, (long long)(L.zero_bytes / 4), 4});
        // outputs: pool -> caller arrays (device) or staging (host)
        char* dst = host ? stage_out + out_off[k] : nullptr;
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
            memcpy(p, j.s0, 8 * nc);
            p += 8 * nc;
            memcpy(p, j.kappa, 8 * nc);
            p += 8 * nc;
            memcpy(p, j.x0, 12 * nb);
            p += 12 * nb;
            if (j.v0) memcpy(p, j.v0, 12 * nb);
        }
    }

    int rc = [&]() -> int {
        SCK(cudaMemcpyAsync(dm, hm, o_cnt, cudaMemcpyHostToDevice, st));
        if (host) SCK(cudaMemcpyAsync(stage_in, srv->pin_in.p, in_bytes, cudaMemcpyHostToDevice, st));
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
        if (host) SCK(cudaMemcpyAsync(srv->pin_out.p, stage_out, out_bytes, cudaMemcpyDeviceToHost, st));
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
