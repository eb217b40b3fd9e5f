// rid_api.cu -- host side of librid: argument checking, device-resident
// system / ensemble / walker state, and the step loop that drives the kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cstdlib>

#include <cudaTypedefs.h>
#include <algorithm>

#include "rid_batch.cuh"
#include "rid_internal.cuh"
#include "rid_tc.cuh"

// ---------------------------------------------------------------------------
// errors
static thread_local std::string g_err = "";

static int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

// The same message store for entry points defined in other translation units.
int rid_fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(e_ == cudaErrorMemoryAllocation ? RID_ERR_OOM : RID_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                     \
    } while (0)

#define TRY(expr)                       \
    do {                                \
        int r_ = (expr);                \
        if (r_ != RID_OK) return r_;    \
    } while (0)

// A grow-only device buffer.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    int ensure(size_t n) {
        if (n <= bytes) return RID_OK;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        if (n == 0) return RID_OK;
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            return fail(RID_ERR_OOM, "cudaMalloc(%zu) failed: %s", n, cudaGetErrorString(e));
        }
        bytes = n;
        return RID_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

// The pre-swizzled BF16 weight image and its tensor maps.
struct TcVariant {
    bool ok = false;
    int stages = 0, Kpmax = 0, tmem_cols = 0, nacc = 1, acc_cols = 0;
    int max_stages = 0, tuned_W = -1;   // weight-stage depth: chosen by timing at each new walker count
    unsigned stage_bytes = 0;
    long long member_rows = 0;
    long long grow[2 * RID_MAX_LAYERS] = {0};
    int gN[2 * RID_MAX_LAYERS] = {0}, gKp[2 * RID_MAX_LAYERS] = {0}, geb[2 * RID_MAX_LAYERS] = {0};
    DevBuf blob, wscale;
    CUtensorMap big{}, small{};
    // cluster variant (k_mlp_tc_cluster): each GEMM's output columns split over
    // csize = 2 or 4 CTAs; index 1 = two CTAs, 2 = four.  The cluster size in use
    // is chosen by timing the force evaluation at each new walker count.
    bool cl_ok[3] = {false, false, false};
    int cl_stages[3] = {0, 0, 0}, cl_acc_cols[3] = {0, 0, 0}, cl_tmem_cols[3] = {0, 0, 0};
    unsigned cl_stage_bytes[3] = {0, 0, 0};
    int csize = 1, cs_W = -1;
    int used_cs = 0;   // cluster size of the last launch (0: none yet)
    // small-batch kernel (k_mlp_tc_small): [k][cs], k = 0, 1, 2 for 16, 32, 64
    // MMA columns, cs = 1..4 CTAs per member splitting the 128-output tiles
    int s_tiles = 0;   // 128-output tiles of the widest GEMM
    bool s_ok[3][5] = {};
    int s_stages[3][5] = {}, s_acc_cols[3][5] = {}, s_tmem_cols[3][5] = {}, s_nacc[3][5] = {};
};

struct rid_system {
    rid_system_desc desc{};
    SysDev S{};
    int device = 0;
    DevBuf d_dih, d_cv, d_acv_off, d_acv, d_cvdist;
    bool has_dist = false;     // some CV is a distance (cv_atoms row (a, b, -1, -1))
    // ensemble
    bool has_ens = false;
    EnsDev E{};
    int precision = RID_PREC_FP32;
    DevBuf d_W, d_WT, d_b, d_wout, d_bout;
    TcVariant tcv;
    int Dp = 0;
    DevBuf tsave, rsave, qsave, d_err;   // rsave: FP32 residual stream of the tensor-core kernel (resnet)
    // state
    int cap = 0;
    DevBuf x, v, f, fff, s, J, u, gradA, Aval, eps, hs, eff, flags;
    // label
    DevBuf lsum, lsum2, lbsum, ls0, lkap;
    DevBuf lfused;   // rid_label through the persistent label kernel: its job, items and counter
    // staging for host I/O and traces
    DevBuf io0, io1, tr_cv, tr_eps, tr_en, tr_chunk, out_mf, out_se, out_sd;
    // resident walker session
    int W_act = 0;
    uint64_t step_next = 0;
    bool loaded = false;
    bool pending = false;      // the last step's closing half (finish + kick) is still to run
    // graph replay: the Philox step index is read from a device base
    DevBuf d_stepbase;
    bool graph_mode = false;
    bool tuning = false;       // inside the cluster-size tuner
    int cs_force = 0;          // cluster size fixed by rid_set_mlp_cluster (0: tuned)
    // force-field CTA size: tuned at each new walker count (ff_W), or fixed
    int ff_th = 0, ff_W = -1, ff_force = 0;
    // run by the request loop: no tuners (their timing syncs would stall the
    // loop, and a choice timed alone is not the one for a shared GPU): one CTA
    // per tile, the default force-field size, the deepest weight ring
    bool serving = false;
    // the force field runs on a side stream, concurrently with the ensemble kernel
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaStream_t cap_stream = nullptr;   // captures the graph of a long run's chunk
    // kernel timing
    bool prof_on = false;
    bool fused_on = true;      // small exploration calls in one persistent launch (rid_set_fused_steps)
    std::vector<std::string> prof_names;
    struct Rec { int id; cudaEvent_t a, b; };
    std::vector<Rec> prof_recs;
    long long launches = 0;
};

// Accessors for the batch / server code in other translation units.
const SysDev* rid_sys_dev(const rid_system* sys) { return &sys->S; }
int rid_sys_device(const rid_system* sys) { return sys->device; }

// Run one kernel launcher, bracketed by events while profiling is enabled.
template <typename F>
static int timed_launch(rid_system* sys, const char* name, cudaStream_t st, F&& launch) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (sys->prof_on) {
        CK(cudaEventCreate(&a));
        CK(cudaEventCreate(&b));
        CK(cudaEventRecord(a, st));
    }
    launch();
    ++sys->launches;
    if (sys->prof_on) {
        CK(cudaEventRecord(b, st));
        int id = -1;
        for (size_t i = 0; i < sys->prof_names.size(); ++i)
            if (sys->prof_names[i] == name) id = (int)i;
        if (id < 0) { id = (int)sys->prof_names.size(); sys->prof_names.push_back(name); }
        sys->prof_recs.push_back({id, a, b});
    }
    return RID_OK;
}

static int check_device(rid_system* sys) {
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != sys->device) return fail(RID_ERR_STATE, "system was created on device %d, current device is %d", sys->device, dev);
    return RID_OK;
}

static StateDev state_view(rid_system* sys) {
    StateDev st{};
    st.W = sys->cap;
    st.x = sys->x.as<float4>();
    st.v = sys->v.as<float4>();
    st.f = sys->f.as<float4>();
    st.fff = sys->fff.as<float4>();
    st.s = sys->s.as<float>();
    st.J = sys->J.as<float4>();
    st.u = sys->u.as<float>();
    st.gradA = sys->gradA.as<float>();
    st.Aval = sys->Aval.as<float>();
    st.eps = sys->eps.as<float>();
    st.hs = sys->hs.as<float>();
    st.eff = sys->eff.as<double>();
    st.flags = sys->flags.as<int>();
    st.stepbase = sys->graph_mode ? sys->d_stepbase.as<uint32_t>() : nullptr;
    return st;
}

// The kernels index per-walker arrays by the walker count of the current call
// (StateDev.W is set to it), so capacity only bounds the allocation.
static int ensure_state(rid_system* sys, int W) {
    const int N = sys->S.N, C = sys->S.C;
    const size_t nb = (size_t)W * N, nc = (size_t)W * C;
    TRY(sys->x.ensure(nb * sizeof(float4)));
    TRY(sys->v.ensure(nb * sizeof(float4)));
    TRY(sys->f.ensure(nb * sizeof(float4)));
    TRY(sys->fff.ensure(nb * sizeof(float4)));
    TRY(sys->s.ensure(nc * sizeof(float)));
    TRY(sys->J.ensure(nc * 4 * sizeof(float4)));
    TRY(sys->u.ensure(nc * 2 * sizeof(float)));
    TRY(sys->eps.ensure((size_t)W * sizeof(float)));
    TRY(sys->eff.ensure((size_t)W * sizeof(double)));
    TRY(sys->flags.ensure((size_t)W * sizeof(int)));
    if (sys->has_ens) {
        const EnsDev& E = sys->E;
        TRY(sys->gradA.ensure((size_t)E.M * nc * sizeof(float)));
        TRY(sys->Aval.ensure((size_t)E.M * W * sizeof(float)));
        TRY(sys->Aval.ensure((size_t)E.M * W * sizeof(float)));
        if (sys->precision == RID_PREC_FP32) {
            TRY(sys->hs.ensure(rid_mlp_fp32_scratch_floats(W, E.M, E.L, E.H) * sizeof(float)));
        } else {
            const size_t ntiles = (size_t)(W + 127) / 128;
            TRY(sys->tsave.ensure((size_t)E.M * ntiles * E.L * 128 * E.H * sizeof(__nv_bfloat16)));
            if (E.resnet) TRY(sys->rsave.ensure((size_t)E.M * ntiles * 128 * E.H * sizeof(float)));
            TRY(sys->qsave.ensure((size_t)E.M * ntiles * TC_MAX_QSLICES * 128 * sizeof(float)));
        }
    }
    if (W > sys->cap) sys->cap = W;
    return RID_OK;
}

// ---------------------------------------------------------------------------
extern "C" int rid_version(void) { return 100; }

extern "C" const char* rid_status_string(int s) {
    switch (s) {
        case RID_OK: return "ok";
        case RID_ERR_ARG: return "invalid argument";
        case RID_ERR_OOM: return "out of device memory";
        case RID_ERR_CUDA: return "CUDA error";
        case RID_ERR_NONFINITE: return "non-finite positions or forces";
        case RID_ERR_TIMEOUT: return "timeout";
        case RID_NOT_READY: return "not ready";
        case RID_ERR_STATE: return "invalid state";
        case RID_ERR_CANCELLED: return "cancelled";
        default: return "unknown status";
    }
}

extern "C" const char* rid_last_error(void) { return g_err.c_str(); }

static void destroy_all(rid_system* sys) {
    DevBuf* bufs[] = {&sys->d_dih, &sys->d_cv, &sys->d_acv_off, &sys->d_acv, &sys->d_cvdist, &sys->d_W, &sys->d_WT, &sys->d_b,
                      &sys->d_wout, &sys->d_bout, &sys->x, &sys->v, &sys->f, &sys->fff, &sys->s, &sys->J,
                      &sys->u, &sys->gradA, &sys->Aval, &sys->eps, &sys->hs, &sys->eff, &sys->flags,
                      &sys->lsum, &sys->lsum2, &sys->lbsum, &sys->ls0, &sys->lkap, &sys->io0, &sys->io1,
                      &sys->tr_cv, &sys->tr_eps, &sys->tr_en, &sys->tr_chunk, &sys->out_mf, &sys->out_se,
                      &sys->out_sd};
    for (DevBuf* b : bufs) b->release();
    sys->tcv.blob.release();
    sys->tsave.release();
    sys->rsave.release();
    sys->qsave.release();
    sys->d_err.release();
    for (auto& r : sys->prof_recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    sys->prof_recs.clear();
    if (sys->ev_fork) cudaEventDestroy(sys->ev_fork);
    if (sys->ev_join) cudaEventDestroy(sys->ev_join);
    if (sys->side) cudaStreamDestroy(sys->side);
    if (sys->cap_stream) cudaStreamDestroy(sys->cap_stream);
    sys->ev_fork = sys->ev_join = nullptr;
    sys->side = sys->cap_stream = nullptr;
}

extern "C" int rid_create_system(const rid_system_desc* d, rid_system** out) {
    if (!d || !out) return fail(RID_ERR_ARG, "NULL argument");
    *out = nullptr;
    const int N = d->n_beads, C = d->n_cv;
    if (N < 4 || N > RID_MAX_BEADS) return fail(RID_ERR_ARG, "n_beads=%d outside [4, %d]", N, RID_MAX_BEADS);
    if (C < 1 || C > RID_MAX_CV) return fail(RID_ERR_ARG, "n_cv=%d outside [1, %d]", C, RID_MAX_CV);
    if (d->output_freq < 1) return fail(RID_ERR_ARG, "output_freq must be >= 1");
    if (d->reserved0 != 0) return fail(RID_ERR_ARG, "reserved0 must be 0");
    if (!(d->mass > 0) || !(d->kT >= 0) || !(d->dt > 0) || !(d->gamma >= 0))
        return fail(RID_ERR_ARG, "need mass > 0, kT >= 0, dt > 0, gamma >= 0");
    if (!(d->lj_rc > 0) || !(d->lj_sigma > 0)) return fail(RID_ERR_ARG, "need lj_rc > 0, lj_sigma > 0");
    if (!d->dihedral_k || !d->dihedral_delta || !d->cv_atoms) return fail(RID_ERR_ARG, "NULL parameter array");
    bool any_dist = false;
    for (int j = 0; j < C; ++j) {
        const int* q = d->cv_atoms + 4 * j;
        const bool dist = q[2] == -1 && q[3] == -1;   // the distance between beads q[0] and q[1]
        any_dist |= dist;
        for (int a = 0; a < (dist ? 2 : 4); ++a)
            if (q[a] < 0 || q[a] >= N) return fail(RID_ERR_ARG, "cv_atoms[%d][%d]=%d outside [0, %d)", j, a, q[a], N);
        if (dist ? q[0] == q[1]
                 : (q[0] == q[1] || q[1] == q[2] || q[2] == q[3] || q[0] == q[2] || q[1] == q[3] || q[0] == q[3]))
            return fail(RID_ERR_ARG, "cv %d has repeated beads", j);
    }
    int dev = 0;
    CK(cudaGetDevice(&dev));
    rid_system* sys = new rid_system();
    sys->device = dev;
    sys->desc = *d;
    sys->desc.dihedral_k = nullptr;
    sys->desc.dihedral_delta = nullptr;
    sys->desc.cv_atoms = nullptr;
    SysDev& S = sys->S;
    S.N = N;
    S.C = C;
    S.output_freq = d->output_freq;
    S.inv_mass = (float)(1.0 / d->mass);
    S.half_dt = (float)(0.5 * d->dt);
    const double c1 = std::exp(-d->gamma * d->dt);
    S.c1 = (float)c1;
    S.c2 = (float)std::sqrt((1.0 - c1 * c1) * d->kT / d->mass);
    S.sd_mb = (float)std::sqrt(d->kT / d->mass);
    S.kb = (float)d->bond_k;
    S.r0 = (float)d->bond_r0;
    S.ka = (float)d->angle_k;
    S.th0 = (float)d->angle_theta0;
    S.lj_eps24 = (float)(24.0 * d->lj_eps);
    S.lj_eps4 = (float)(4.0 * d->lj_eps);
    S.sig2 = (float)(d->lj_sigma * d->lj_sigma);
    S.rc2 = (float)(d->lj_rc * d->lj_rc);
    {
        const double sr6 = std::pow(d->lj_sigma / d->lj_rc, 6.0);
        S.urc = (float)(4.0 * d->lj_eps * (sr6 * sr6 - sr6));
    }
    S.key0 = (uint32_t)d->seed;
    S.key1 = (uint32_t)(d->seed >> 32);
    // parameters
    std::vector<float> dih((size_t)(N - 3) * 6);
    for (int k = 0; k < N - 3; ++k)
        for (int n = 0; n < 3; ++n) {
            dih[6 * k + n] = (float)d->dihedral_k[3 * k + n];
            dih[6 * k + 3 + n] = (float)d->dihedral_delta[3 * k + n];
        }
    // chain-rule list: the (CV, slot) pairs touching each bead, in CV order
    // (a distance CV has two slots; the list is padded to 4 C entries)
    std::vector<int> off(N + 1, 0);
    for (int j = 0; j < C; ++j)
        for (int a = 0; a < 4; ++a)
            if (d->cv_atoms[4 * j + a] >= 0) off[d->cv_atoms[4 * j + a] + 1]++;
    for (int i = 0; i < N; ++i) off[i + 1] += off[i];
    std::vector<int2> acv(4 * C, make_int2(0, 0));
    {
        std::vector<int> fill(off.begin(), off.end() - 1);
        for (int j = 0; j < C; ++j)
            for (int a = 0; a < 4; ++a)
                if (d->cv_atoms[4 * j + a] >= 0) acv[fill[d->cv_atoms[4 * j + a]]++] = make_int2(j, a);
    }
    std::vector<int> cvdist(C);
    for (int j = 0; j < C; ++j) cvdist[j] = d->cv_atoms[4 * j + 2] < 0 ? 1 : 0;
    int r = RID_OK;
    if ((r = sys->d_dih.ensure(dih.size() * sizeof(float))) || (r = sys->d_cv.ensure(C * sizeof(int4))) ||
        (r = sys->d_acv_off.ensure((N + 1) * sizeof(int))) || (r = sys->d_acv.ensure(4 * C * sizeof(int2))) ||
        (r = sys->d_cvdist.ensure(C * sizeof(int)))) {
        destroy_all(sys);
        delete sys;
        return r;
    }
    cudaError_t e = cudaMemcpy(sys->d_dih.p, dih.data(), dih.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(sys->d_cv.p, d->cv_atoms, C * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(sys->d_acv_off.p, off.data(), (N + 1) * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(sys->d_acv.p, acv.data(), 4 * C * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(sys->d_cvdist.p, cvdist.data(), C * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        destroy_all(sys);
        delete sys;
        return fail(RID_ERR_CUDA, "parameter upload failed: %s", cudaGetErrorString(e));
    }
    S.dih = sys->d_dih.as<float>();
    S.cv = sys->d_cv.as<int4>();
    S.acv_off = sys->d_acv_off.as<int>();
    S.acv = sys->d_acv.as<int2>();
    sys->has_dist = any_dist;
    *out = sys;
    return RID_OK;
}

extern "C" int rid_destroy_system(rid_system* sys) {
    if (!sys) return RID_OK;
    destroy_all(sys);
    delete sys;
    return RID_OK;
}

// ---------------------------------------------------------------------------
// BF16 tensor-core path: weight images and tensor maps.
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// FP8 e4m3 (1 sign, 4 exponent bits with bias 7, 3 mantissa bits; no
// infinities; largest finite 448; subnormals k 2^-9): round to nearest even,
// saturating at +-448.
static uint8_t f2e4m3(float f) {
    const uint8_t sgn = std::signbit(f) ? 0x80 : 0x00;
    const double a = std::fabs((double)f);
    if (std::isnan(f)) return sgn | 0x7F;
    if (a >= 448.0) return sgn | 0x7E;
    int e = 0;
    std::frexp(a, &e);                        // a = m 2^e, m in [0.5, 1)
    int E = e - 1;                            // a = (1 + f) 2^E for normal values
    if (a == 0.0 || E < -6) {                 // subnormal range: multiples of 2^-9
        const int q = (int)std::nearbyint(std::ldexp(a, 9));   // q = 8 is the smallest normal, bits 0x08
        return sgn | (uint8_t)q;
    }
    int m = (int)std::nearbyint((std::ldexp(a, -E) - 1.0) * 8.0);
    if (m == 8) { m = 0; ++E; }
    if (E > 8 || (E == 8 && m > 6)) return sgn | 0x7E;
    return sgn | (uint8_t)(((E + 7) << 3) | m);
}

static uint16_t f2bf(float f) {   // round to nearest even
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

static int build_tc_variant(rid_system* sys, const std::vector<float>& W, long long wst, const long long* loff,
                            bool fp8, TcVariant& V) {
    const EnsDev& E = sys->E;
    const int M = E.M, D = E.D, L = E.L, H = E.H, Dp = sys->Dp, G = 2 * L;
    V.ok = false;
    int nmax = 0, rowbytes = 0;
    long long rows = 0;
    for (int g = 0; g < G; ++g) {
        const bool fwd = g < L;
        const int l = fwd ? g : G - 1 - g;
        V.geb[g] = (fp8 && fwd) ? 1 : 2;
        const int kc = 128 / V.geb[g];            // columns per 128-byte K-chunk
        V.gN[g] = fwd ? H : (l == 0 ? Dp : H);
        V.gKp[g] = (((fwd ? (l == 0 ? D : H) : H) + kc - 1) / kc) * kc;
        if (V.gN[g] > nmax) nmax = V.gN[g];
        if (V.gKp[g] * V.geb[g] > rowbytes) rowbytes = V.gKp[g] * V.geb[g];
        V.grow[g] = rows;
        rows += (long long)(V.gKp[g] * V.geb[g] / 128) * V.gN[g];
    }
    if (rowbytes / 128 > TC_MAX_KCHUNKS) return fail(RID_ERR_ARG, "tensor-core path: K up to %d", 64 * TC_MAX_KCHUNKS);
    V.Kpmax = rowbytes / 2;
    V.member_rows = rows;
    V.stage_bytes = (unsigned)(nmax < 256 ? nmax : 256) * 128u;
    const size_t fixed = 1024 + (size_t)V.Kpmax * 256u + sizeof(float) * (size_t)(L + 1) * H;
    const size_t budget = 225u * 1024u;
    if (fixed + 2 * (size_t)V.stage_bytes > budget)
        return fail(RID_ERR_ARG, "tensor-core path: tile too large for shared memory");
    V.stages = (int)((budget - fixed) / V.stage_bytes);
    if (V.stages > TC_MAX_STAGES) V.stages = TC_MAX_STAGES;
    V.max_stages = V.stages;
    V.tuned_W = -1;
    V.acc_cols = (nmax + 31) / 32 * 32;
    V.nacc = 2 * V.acc_cols <= 512 ? 2 : 1;
    V.tmem_cols = 32;
    while (V.tmem_cols < V.nacc * V.acc_cols) V.tmem_cols *= 2;
    // cluster variants: two operand buffers, each CTA streams n_s = N / S
    // (rounded up to 16) rows of every weight chunk
    for (int k = 1; k <= 2; ++k) {
        const int cs = 1 << k;
        int nsl = 0;
        for (int g = 0; g < G; ++g) {
            const int ns = ((V.gN[g] + cs - 1) / cs + 15) / 16 * 16;
            if (ns > nsl) nsl = ns;
        }
        const size_t fixc = 1024 + 2 * (size_t)V.Kpmax * 256u + sizeof(float) * (size_t)(L + 1) * H;
        const unsigned sb = (unsigned)nsl * 128u;
        V.cl_ok[k] = fixc + 2 * (size_t)sb <= budget && nsl <= 256;
        if (!V.cl_ok[k]) continue;
        V.cl_stage_bytes[k] = sb;
        V.cl_stages[k] = (int)std::min<size_t>((budget - fixc) / sb, TC_MAX_STAGES);
        V.cl_acc_cols[k] = (nsl + 31) / 32 * 32;
        V.cl_tmem_cols[k] = 32;
        while (V.cl_tmem_cols[k] < 2 * V.cl_acc_cols[k]) V.cl_tmem_cols[k] *= 2;
    }
    // small-batch variants (BF16 only: the transposed GEMMs take the forward
    // weights as the A operand in their BF16 image), per MMA width and number
    // of CTAs splitting the 128-output tiles
    int nmx = 0;
    for (int g = 0; g < G; ++g) nmx = std::max(nmx, (V.gN[g] + 127) / 128);
    V.s_tiles = nmx;
    for (int k = 0; k < 3; ++k)
        for (int cs = 1; cs <= 4; ++cs) {
            const int nw = 16 << k, own = (nmx + cs - 1) / cs;
            TcArgs Q{};
            Q.L = L;
            Q.H = H;
            Q.Kpmax = V.Kpmax;
            Q.resnet = sys->E.resnet;
            Q.csize = cs;
            Q.stages = 0;
            for (int g = 0; g < G; ++g) Q.gN[g] = V.gN[g];
            const size_t fixs = rid_mlp_tc_small_smem_bytes(Q, nw);
            const int acc = (own * nw + 31) / 32 * 32;
            V.s_nacc[k][cs] = 2 * acc <= 512 ? 2 : 1;
            V.s_acc_cols[k][cs] = acc;
            V.s_tmem_cols[k][cs] = 32;
            while (V.s_tmem_cols[k][cs] < V.s_nacc[k][cs] * acc) V.s_tmem_cols[k][cs] *= 2;
            V.s_stages[k][cs] =
                fixs + 2 * 16384 <= budget ? (int)std::min<size_t>((budget - fixs) / 16384, TC_MAX_STAGES) : 0;
            // (the kernel is built for 16 MMA columns only)
            V.s_ok[k][cs] = k == 0 && !fp8 && nmx <= 4 && cs <= nmx && acc <= 512 && V.s_stages[k][cs] >= 2;
        }
    V.cs_W = -1;
    V.csize = 1;
    // pre-swizzled byte image: per GEMM, per 128-byte K-chunk, N rows of 128 bytes
    std::vector<uint8_t> img((size_t)M * rows * 128, 0);
    std::vector<float> scale((size_t)M * G, 1.0f);
    for (int m = 0; m < M; ++m)
        for (int g = 0; g < G; ++g) {
            const bool fwd = g < L;
            const int l = fwd ? g : G - 1 - g;
            const int fin = l == 0 ? D : H;
            const float* Wl = W.data() + (size_t)m * wst + loff[l];   // [H][fin]
            const int N = V.gN[g], eb = V.geb[g], kc = 128 / eb;
            float s = 1.0f;
            if (eb == 1) {
                float amax = 0.0f;
                for (size_t i = 0; i < (size_t)H * fin; ++i) amax = std::max(amax, std::fabs(Wl[i]));
                s = amax > 0.0f ? amax / 448.0f : 1.0f;
                scale[(size_t)m * G + g] = s;
            }
            for (int c = 0; c < V.gKp[g] / kc; ++c) {
                const size_t base = ((size_t)m * rows + V.grow[g] + (size_t)c * N) * 128;
                for (int n = 0; n < N; ++n)
                    for (int kl = 0; kl < kc; ++kl) {
                        const int k = c * kc + kl;
                        float val = 0.0f;
                        if (fwd) { if (k < fin) val = Wl[(size_t)n * fin + k]; }      // W_l[n][k]
                        else if (n < fin && k < H) val = Wl[(size_t)k * fin + n];     // W_l^T[n][k]
                        const int byte = kl * eb;
                        const int j = (byte >> 4) ^ (n & 7);
                        uint8_t* dst = img.data() + base + (size_t)n * 128 + j * 16 + (byte & 15);
                        if (eb == 1) {
                            dst[0] = f2e4m3(val / s);
                        } else {
                            const uint16_t h = f2bf(val);
                            dst[0] = (uint8_t)(h & 0xFF);
                            dst[1] = (uint8_t)(h >> 8);
                        }
                    }
            }
        }
    TRY(V.blob.ensure(img.size()));
    CK(cudaMemcpy(V.blob.p, img.data(), img.size(), cudaMemcpyHostToDevice));
    TRY(V.wscale.ensure(scale.size() * sizeof(float)));
    CK(cudaMemcpy(V.wscale.p, scale.data(), scale.size() * sizeof(float), cudaMemcpyHostToDevice));
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return fail(RID_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the CUDA driver");
    const cuuint64_t dims[2] = {128, (cuuint64_t)M * rows};
    const cuuint64_t strides[1] = {128};
    const cuuint32_t estr[2] = {1, 1};
    const cuuint32_t box_big[2] = {128, 64}, box_small[2] = {128, 8};
    CUresult r1 = enc(&V.big, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, V.blob.p, dims, strides, box_big, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    CUresult r2 = enc(&V.small, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, V.blob.p, dims, strides, box_small, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS)
        return fail(RID_ERR_CUDA, "tensor map encoding failed (%d, %d)", (int)r1, (int)r2);
    V.ok = true;
    return RID_OK;
}

extern "C" int rid_set_ensemble(rid_system* sys, const rid_ensemble_desc* d) {
    if (!sys || !d || !d->weights) return fail(RID_ERR_ARG, "NULL argument");
    TRY(check_device(sys));
    const int M = d->n_models, D = d->n_in, L = d->n_layers, Hu = d->width;
    if (M < 1 || M > RID_MAX_MODELS) return fail(RID_ERR_ARG, "n_models=%d outside [1, %d]", M, RID_MAX_MODELS);
    if (D != 2 * sys->S.C) return fail(RID_ERR_ARG, "n_in=%d must equal 2 * n_cv = %d", D, 2 * sys->S.C);
    if (L < 1 || L > RID_MAX_LAYERS) return fail(RID_ERR_ARG, "n_layers=%d outside [1, %d]", L, RID_MAX_LAYERS);
    if (Hu < 1 || Hu > RID_MAX_WIDTH) return fail(RID_ERR_ARG, "width=%d outside [1, %d]", Hu, RID_MAX_WIDTH);
    if (d->precision != RID_PREC_FP32 && d->precision != RID_PREC_BF16 && d->precision != RID_PREC_FP8)
        return fail(RID_ERR_ARG, "unknown precision %d", d->precision);
    if (!(d->trust_lo < d->trust_hi)) return fail(RID_ERR_ARG, "need trust_lo < trust_hi");
    // The kernels tile the hidden width in multiples of 32.  A width that is
    // not one is padded with hidden units whose incoming weights, bias and
    // outgoing weights are all zero: such a unit computes tanh(0) = 0 (plus a
    // zero residual), contributes nothing to A and receives a zero gradient,
    // so the padded network is the same function with the same input
    // gradient, exactly.
    const int H = (Hu + 31) / 32 * 32;
    const long long P = (long long)Hu * D + Hu + (long long)(L - 1) * ((long long)Hu * Hu + Hu) + Hu + 1;
    // split the packed layout into W (row-major [H][fin]), W^T, biases, w_out, b_out
    long long wst = (long long)H * D + (long long)(L - 1) * H * H;
    std::vector<float> W((size_t)M * wst, 0.0f), WT((size_t)M * wst, 0.0f), b((size_t)M * L * H, 0.0f),
        wo((size_t)M * H, 0.0f), bo(M);
    long long loff[RID_MAX_LAYERS] = {0};
    for (int l = 1; l < L; ++l) loff[l] = loff[l - 1] + (long long)H * (l == 1 ? D : H);
    for (int m = 0; m < M; ++m) {
        const float* p = d->weights + (size_t)m * P;
        for (int l = 0; l < L; ++l) {
            const int fin = l == 0 ? D : H, finu = l == 0 ? D : Hu;
            float* Wm = W.data() + (size_t)m * wst + loff[l];
            float* WTm = WT.data() + (size_t)m * wst + loff[l];
            for (int o = 0; o < Hu; ++o)
                for (int i = 0; i < finu; ++i) {
                    const float val = p[(size_t)o * finu + i];
                    if (!std::isfinite(val)) return fail(RID_ERR_ARG, "non-finite weight in model %d", m);
                    Wm[(size_t)o * fin + i] = val;
                    WTm[(size_t)i * H + o] = val;
                }
            p += (size_t)Hu * finu;
            for (int o = 0; o < Hu; ++o) b[((size_t)m * L + l) * H + o] = p[o];
            p += Hu;
        }
        for (int o = 0; o < Hu; ++o) wo[(size_t)m * H + o] = p[o];
        bo[m] = p[Hu];
    }
    TRY(sys->d_W.ensure(W.size() * sizeof(float)));
    TRY(sys->d_WT.ensure(WT.size() * sizeof(float)));
    TRY(sys->d_b.ensure(b.size() * sizeof(float)));
    TRY(sys->d_wout.ensure(wo.size() * sizeof(float)));
    TRY(sys->d_bout.ensure(bo.size() * sizeof(float)));
    CK(cudaMemcpy(sys->d_W.p, W.data(), W.size() * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(sys->d_WT.p, WT.data(), WT.size() * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(sys->d_b.p, b.data(), b.size() * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(sys->d_wout.p, wo.data(), wo.size() * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(sys->d_bout.p, bo.data(), bo.size() * sizeof(float), cudaMemcpyHostToDevice));
    EnsDev& E = sys->E;
    E.M = M; E.D = D; E.L = L; E.H = H; E.resnet = d->resnet ? 1 : 0;
    E.e0 = (float)d->trust_lo;
    E.e1 = (float)d->trust_hi;
    E.W = sys->d_W.as<float>();
    E.WT = sys->d_WT.as<float>();
    E.b = sys->d_b.as<float>();
    E.wout = sys->d_wout.as<float>();
    E.bout = sys->d_bout.as<float>();
    E.wstride = wst;
    for (int l = 0; l < RID_MAX_LAYERS; ++l) E.loff[l] = loff[l];
    E.cvdist = sys->has_dist ? sys->d_cvdist.as<int>() : nullptr;
    sys->precision = d->precision;
    sys->has_ens = true;
    E.aslices = 1;
    if (d->precision != RID_PREC_FP32) {
        sys->Dp = (D + 63) / 64 * 64;
        TRY(build_tc_variant(sys, W, wst, loff, d->precision == RID_PREC_FP8, sys->tcv));
        TRY(sys->d_err.ensure(sizeof(int)));
        CK(cudaMemset(sys->d_err.p, 0, sizeof(int)));
    }
    // re-size the ensemble scratch for the current capacity
    if (sys->cap > 0) {
        const int cap = sys->cap;
        sys->cap = 0;
        TRY(ensure_state(sys, cap));
    }
    return RID_OK;
}

// ---------------------------------------------------------------------------
// I/O helpers: bring [W][N][3] float arrays in / out of the float4 state.
static int load_xyz(rid_system* sys, const float* src, float4* dst, long long n, int mem, cudaStream_t st) {
    const float* dsrc = src;
    if (mem == RID_MEM_HOST) {
        TRY(sys->io0.ensure((size_t)n * 3 * sizeof(float)));
        CK(cudaMemcpyAsync(sys->io0.p, src, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, st));
        dsrc = sys->io0.as<float>();
    }
    rid_launch_pack(dsrc, dst, n, st);
    CK(cudaGetLastError());
    return RID_OK;
}

static int store_xyz(rid_system* sys, const float4* src, float* dst, long long n, int mem, cudaStream_t st) {
    if (!dst) return RID_OK;
    float* ddst = dst;
    if (mem == RID_MEM_HOST) {
        TRY(sys->io1.ensure((size_t)n * 3 * sizeof(float)));
        ddst = sys->io1.as<float>();
    }
    rid_launch_unpack(src, ddst, n, st);
    CK(cudaGetLastError());
    if (mem == RID_MEM_HOST) CK(cudaMemcpyAsync(dst, ddst, (size_t)n * 3 * sizeof(float), cudaMemcpyDeviceToHost, st));
    return RID_OK;
}

static int fetch_flags(rid_system* sys, int W, cudaStream_t st, bool* any) {
    std::vector<int> h(W);
    CK(cudaMemcpyAsync(h.data(), sys->flags.p, (size_t)W * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *any = false;
    for (int i = 0; i < W; ++i) *any |= h[i] != 0;
    if (sys->d_err.p) {
        int e = 0;
        CK(cudaMemcpy(&e, sys->d_err.p, sizeof(int), cudaMemcpyDeviceToHost));
        if (e) {
            cudaMemset(sys->d_err.p, 0, sizeof(int));
            return fail(RID_ERR_TIMEOUT, "tensor-core MLP kernel: a bounded wait expired (code %d)", e);
        }
    }
    return RID_OK;
}

static int launch_mlp(rid_system* sys, int W, int mode, StateDev sd, cudaStream_t st, bool values_only = false);

// Side stream (lowest priority) and fork / join events, created on first use.
static int ensure_side(rid_system* sys) {
    if (sys->side) return RID_OK;
    int lo = 0, hi = 0;
    CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    CK(cudaStreamCreateWithPriority(&sys->side, cudaStreamNonBlocking, lo));
    CK(cudaEventCreateWithFlags(&sys->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&sys->ev_join, cudaEventDisableTiming));
    return RID_OK;
}

// Force-field and ensemble kernels at the current positions (the CVs and the
// MLP input have been written by the preceding k_head).  Both depend only on
// the positions: the ensemble kernel (a few CTAs that each need most of an
// SM's shared memory) is launched first on the caller's stream so that it is
// dispatched as soon as k_head ends, and the force field runs concurrently on
// a side stream over the remaining SMs; the caller's stream then waits for it.
static int tune_cluster(rid_system* sys, int W, bool energy, cudaStream_t st);

// The small-batch ensemble kernel's variant for W walkers (0, 1, 2: 16, 32, 64
// MMA columns), or -1 when the batch is larger or the variant does not fit.
// Chosen by walker count alone, never by timing.
// Its CTAs per member: one per 128-output tile of the widest GEMM (up to 4),
// or at most the size fixed by rid_set_mlp_cluster.  Every size gives the
// same bits.
static int small_cs(const rid_system* sys) {
    const int t = std::max(1, sys->tcv.s_tiles);
    return sys->cs_force ? std::min(sys->cs_force, t) : std::min(t, 4);
}
static int small_variant(const rid_system* sys, int W) {
    // 16 MMA columns only: a tcgen05.mma costs about the same whatever its N,
    // so the transposed form pays more MMAs per GEMM (one per 128 outputs
    // instead of per 256) and wins only while its epilogue is much smaller
    // (measured with one CTA per member: the paper's 4 x [300]^4 network at
    // 12 walkers 64 us against 84 us for the row kernel; at 64 walkers 134 us
    // against 84)
    if (sys->precision != RID_PREC_BF16 || W > 16) return -1;
    return sys->tcv.s_ok[0][small_cs(sys)] ? 0 : -1;
}


// Autotuner of the force field's CTA size (threads per walker CTA, hence
// beads per pass and CTAs per SM): at the first force evaluation with a new
// walker count, k_ff alone is timed with every multiple of 32 from 64 up to
// its default (one warm-up and three timed launches each) and the fastest is
// kept, the default unless another is 2% faster.  The forces are the same bits
// with every size.  Skipped while the stream is being captured.
static int tune_ff(rid_system* sys, int W, cudaStream_t st) {
    const int dth = rid_ff_default_threads(sys->S.N);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cs));
    sys->ff_W = W;
    sys->ff_th = dth;
    if (cs != cudaStreamCaptureStatusNone || dth <= 64 || sys->serving) return RID_OK;
    StateDev sd = state_view(sys);
    sd.W = W;
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    float best = 1e30f, tdef = 1e30f;
    int pick = dth;
    for (int th = dth; th >= 64; th -= 32) {
        rid_launch_ff(sys->S, sd, W, false, st, th);
        CK(cudaEventRecord(a, st));
        for (int r = 0; r < 3; ++r) rid_launch_ff(sys->S, sd, W, false, st, th);
        CK(cudaEventRecord(b, st));
        CK(cudaEventSynchronize(b));
        CK(cudaGetLastError());
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, a, b));
        if (th == dth) tdef = ms;
        if (ms < best) {
            best = ms;
            pick = th;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    sys->launches += 4 * ((dth - 64) / 32 + 1);
    sys->ff_th = best < 0.98f * tdef ? pick : dth;
    return RID_OK;
}

static int launch_forces(rid_system* sys, int W, int mode, bool energy, cudaStream_t st) {
    StateDev sd = state_view(sys);
    sd.W = W;
    if (sys->ff_W != W && !sys->tuning && !sys->ff_force) TRY(tune_ff(sys, W, st));
    const int ffth = sys->ff_force ? sys->ff_force : sys->ff_th;
    if (mode == 1 && sys->precision != RID_PREC_FP32 && sys->tcv.cs_W != W && !sys->tuning && !sys->cs_force &&
        small_variant(sys, W) < 0)
        TRY(tune_cluster(sys, W, energy, st));
    if (mode != 1) {
        TRY(timed_launch(sys, "k_ff", st, [&] { rid_launch_ff(sys->S, sd, W, energy, st, ffth); }));
        CK(cudaGetLastError());
        return RID_OK;
    }
    TRY(ensure_side(sys));
    CK(cudaEventRecord(sys->ev_fork, st));
    CK(cudaStreamWaitEvent(sys->side, sys->ev_fork, 0));
    TRY(launch_mlp(sys, W, mode, sd, st));
    cudaStream_t fs = sys->side;
    TRY(timed_launch(sys, "k_ff", fs, [&] { rid_launch_ff(sys->S, sd, W, energy, fs, ffth); }));
    CK(cudaEventRecord(sys->ev_join, fs));
    CK(cudaStreamWaitEvent(st, sys->ev_join, 0));
    CK(cudaGetLastError());
    return RID_OK;
}

// The one-CTA ensemble kernel: chunk-interleaved epilogue when the TMEM
// accumulator is double buffered (width <= 256), the contiguous-column
// epilogue of k_mlp_tc_wide when a single accumulator fills TMEM.
static cudaError_t launch_tc1(const TcArgs& P, const TcVariant& V, cudaStream_t st) {
    return V.nacc == 1 ? rid_launch_mlp_tc_wide(P, V.big, V.small, st) : rid_launch_mlp_tc(P, V.big, V.small, st);
}

// Cluster size used before the tuner has timed a walker count: the largest
// of 4 and 2 whose grid (tiles x members x size) still fits the 152 SMs once,
// else 1 (k_mlp_tc, one CTA per tile and member).
static int default_cluster(const TcVariant& V, int ctas) {
    if (V.cl_ok[2] && ctas * 4 <= 152) return 4;
    if (V.cl_ok[1] && ctas * 2 <= 152) return 2;
    return 1;
}

// Autotuner of the ensemble kernel's cluster size: at the first ensemble
// force evaluation with a new walker count, the whole concurrent phase (the
// ensemble kernel on the caller's stream, the force field beside it) is timed
// with each eligible cluster size (1, 2, 4; one warm-up and three timed
// evaluations each) and the fastest is kept.  Splitting the columns over more
// CTAs shortens the ensemble's chain but takes SMs from the force field, so
// the choice is made on the phase, not on the ensemble kernel alone.  Every
// candidate computes the same quantities; the outputs of the last evaluation
// are the ones left in place.  Skipped while the stream is being captured.
static int tune_cluster(rid_system* sys, int W, bool energy, cudaStream_t st) {
    TcVariant& V = sys->tcv;
    const int ctas = (W + 127) / 128 * sys->E.M;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cs));
    std::vector<int> cand = {1};
    if (V.cl_ok[1]) cand.push_back(2);
    if (V.cl_ok[2]) cand.push_back(4);
    if (sys->serving) {
        V.csize = 1;
        V.cs_W = W;
        return RID_OK;
    }
    if (cs != cudaStreamCaptureStatusNone || cand.size() == 1) {
        V.csize = cs != cudaStreamCaptureStatusNone ? default_cluster(V, ctas) : 1;
        V.cs_W = W;
        return RID_OK;
    }
    sys->tuning = true;
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    float best = 1e30f;
    int pick = 1;
    for (int c : cand) {
        V.csize = c;
        V.cs_W = W;
        int rc = launch_forces(sys, W, 1, energy, st);
        if (rc == RID_OK) {
            CK(cudaEventRecord(a, st));
            for (int r = 0; r < 3 && rc == RID_OK; ++r) rc = launch_forces(sys, W, 1, energy, st);
            CK(cudaEventRecord(b, st));
        }
        if (rc != RID_OK) {
            sys->tuning = false;
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            return rc;
        }
        CK(cudaEventSynchronize(b));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, a, b));
        if (ms < best) {
            best = ms;
            pick = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    sys->tuning = false;
    V.csize = pick;
    V.cs_W = W;
    return RID_OK;
}

// Autotuner of the tensor-core kernel's weight pipeline: at the first
// evaluation with a new walker count, time the kernel with 2, 3, 4, ... up
// to the largest stage ring that fits shared memory (three launches each,
// after one warm-up) and keep the fastest.  Results do not depend on the
// choice.  Skipped while the stream is being captured.
static int tune_tc_stages(rid_system* sys, TcArgs P, cudaStream_t st) {
    TcVariant& V = sys->tcv;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone || V.max_stages <= 2 || sys->serving) {
        V.tuned_W = P.W;
        return RID_OK;
    }
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    float best = 1e30f;
    int pick = V.max_stages;
    for (int ns = 2; ns <= V.max_stages; ++ns) {
        P.stages = ns;
        CK(launch_tc1(P, V, st));
        CK(cudaEventRecord(a, st));
        for (int r = 0; r < 3; ++r) CK(launch_tc1(P, V, st));
        CK(cudaEventRecord(b, st));
        CK(cudaEventSynchronize(b));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, a, b));
        if (ms < best * 0.98f) {        // prefer fewer stages unless clearly slower
            best = ms;
            pick = ns;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    V.stages = pick;
    V.tuned_W = P.W;
    sys->launches += 4 * (V.max_stages - 1);
    return RID_OK;
}

// values_only: the member values alone (the tensor-core kernel then runs the
// L forward GEMMs and skips the input gradient; the FP32 kernel forms both).
static int launch_mlp(rid_system* sys, int W, int mode, StateDev sd, cudaStream_t st, bool values_only) {
    EnsDev& E = sys->E;
    if (mode == 1 && sys->precision != RID_PREC_FP32) {
        const TcVariant& V = sys->tcv;
        TcArgs P{};
        P.W = W; P.C = sys->S.C; P.D = E.D; P.Dp = sys->Dp; P.L = E.L; P.H = E.H; P.M = E.M;
        P.stages = V.stages; P.Kpmax = V.Kpmax; P.ntiles = (W + 127) / 128;
        P.tmem_cols = V.tmem_cols; P.nacc = V.nacc; P.acc_cols = V.acc_cols; P.stage_bytes = V.stage_bytes;
        P.u = sd.u; P.bias = E.b; P.wout = E.wout; P.bout = E.bout; P.cvdist = E.cvdist;
        P.tsave = sys->tsave.as<__nv_bfloat16>(); P.gradA = sd.gradA; P.Apart = sd.Aval; P.err = sys->d_err.as<int>();
        P.member_rows = V.member_rows;
        for (int g = 0; g < 2 * E.L; ++g) {
            P.grow[g] = V.grow[g];
            P.gN[g] = V.gN[g];
            P.gKp[g] = V.gKp[g];
            P.geb[g] = V.geb[g];
        }
        P.wscale = V.wscale.as<float>();
        P.resnet = E.resnet;
        P.qsave = sys->qsave.as<float>();
        P.rsave = E.resnet ? sys->rsave.as<float>() : nullptr;
        P.ngemm = values_only ? E.L : 2 * E.L;
        cudaError_t le = cudaSuccess;
        const int sk = small_variant(sys, W);
        if (sk >= 0 && !values_only) {
            // up to 16 walkers: the transposed small-batch kernel, its output tiles split over a cluster
            // while a server runs a job on the system, the lean variant: 8 epilogue warps and
            // 3 weight stages, so that its CTAs can share SMs with the other jobs' kernels
            const int nw = 16 << sk, scs = small_cs(sys);
            const int epi = sys->serving ? 8 : 16;
            P.stages = sys->serving ? std::min(3, V.s_stages[sk][scs]) : V.s_stages[sk][scs];
            P.acc_cols = V.s_acc_cols[sk][scs];
            P.tmem_cols = V.s_tmem_cols[sk][scs];
            P.nacc = V.s_nacc[sk][scs];
            P.csize = scs;
            sys->tcv.used_cs = scs;
            TRY(timed_launch(sys, "k_mlp_tc", st, [&] { le = rid_launch_mlp_tc_small(P, V.big, V.small, nw, epi, st); }));
            if (le != cudaSuccess) return fail(RID_ERR_CUDA, "k_mlp_tc_small launch: %s", cudaGetErrorString(le));
            E.aslices = 1;
            return RID_OK;
        }
        const int cs = sys->cs_force ? sys->cs_force : V.cs_W == W ? V.csize : default_cluster(V, P.ntiles * E.M);
        if (cs > 1 && !V.cl_ok[cs == 2 ? 1 : 2])
            return fail(RID_ERR_ARG, "ensemble kernel: cluster size %d does not fit this ensemble's shape", cs);
        sys->tcv.used_cs = cs;
        if (cs == 1) {
            if (V.tuned_W != W) TRY(tune_tc_stages(sys, P, st));
            P.stages = V.stages;
            P.csize = 1;
            TRY(timed_launch(sys, "k_mlp_tc", st, [&] { le = launch_tc1(P, V, st); }));
        } else {
            const int k = cs == 2 ? 1 : 2;
            P.csize = cs;
            P.stages = V.cl_stages[k];
            P.stage_bytes = V.cl_stage_bytes[k];
            P.acc_cols = V.cl_acc_cols[k];
            P.tmem_cols = V.cl_tmem_cols[k];
            P.nacc = 2;
            TRY(timed_launch(sys, "k_mlp_tc", st, [&] { le = rid_launch_mlp_tc_cluster(P, V.big, V.small, st); }));
        }
        if (le != cudaSuccess) return fail(RID_ERR_CUDA, "k_mlp_tc launch: %s", cudaGetErrorString(le));
        E.aslices = 1;
    } else if (mode == 1) {
        E.aslices = 1;
        TRY(timed_launch(sys, "k_mlp_fp32", st, [&] { rid_launch_mlp_fp32(E, sd, W, sys->S.C, st); }));
    }
    return RID_OK;
}

// k_head: finish the previous evaluation and / or open the next step.
static int launch_head(rid_system* sys, int W, int mode, const LabelDev* lab, bool fin, bool kick, int integ,
                       long long t_fin, int slot, float* cv, float* eps, double* en, long long T, uint32_t step,
                       cudaStream_t st) {
    HeadArgs a{};
    a.S = sys->S;
    a.st = state_view(sys);
    a.st.W = W;
    if (mode == 1) a.E = sys->E;
    if (lab) a.lab = *lab;
    a.W = W;
    a.mode = mode;
    a.fin = fin;
    a.kick = kick;
    a.integ = integ;
    a.no_split = sys->serving;
    a.t_fin = t_fin;
    a.slot = fin ? slot : -1;
    a.cv_out = cv;
    a.eps_out = eps;
    a.energy_out = en;
    a.energy = fin && en != nullptr && slot >= 0;
    a.T = T;
    a.step = step;
    TRY(timed_launch(sys, "k_head", st, [&] { rid_launch_head(a, st); }));
    CK(cudaGetLastError());
    return RID_OK;
}

// Evaluate the total force at the current positions (no step): CVs, force
// field, ensemble, then the finish that stores f.
static int evaluate_at_rest(rid_system* sys, int W, int mode, const LabelDev* lab, cudaStream_t st) {
    TRY(launch_head(sys, W, mode, lab, false, false, 1, -1, -1, nullptr, nullptr, nullptr, 0, 0, st));
    TRY(launch_forces(sys, W, mode, false, st));
    TRY(launch_head(sys, W, mode, lab, true, false, 0, -1, -1, nullptr, nullptr, nullptr, 0, 0, st));
    return RID_OK;
}

// n_steps BAOAB steps.  On entry either f is stored for the current x
// (pending = false) or the closing half of the previous step is still to run
// (pending = true, its forces and CVs are in the buffers).  The closing half of
// the last step is run here only if it carries a trace or label sample
// (close_last), else it is left pending for the next call or read.
static int run_steps(rid_system* sys, int W, int mode, const LabelDev* lab, int64_t n_steps, uint64_t step0,
                     float* cv, float* eps, double* en, long long T, bool& pending, bool close_last, cudaStream_t st) {
    const int of = sys->S.output_freq;
    auto slot_of = [&](long long t) { return ((t + 1) % of == 0) ? (int)((t + 1) / of - 1) : -1; };
    for (long long t = 0; t < n_steps; ++t) {
        const bool fin = t > 0 || pending;
        TRY(launch_head(sys, W, mode, lab, fin, true, 2, t - 1, t > 0 ? slot_of(t - 1) : -1, cv, eps, en, T,
                        (uint32_t)(step0 + t), st));
        TRY(launch_forces(sys, W, mode, en != nullptr && slot_of(t) >= 0, st));
        pending = true;
    }
    const bool need = n_steps > 0 && (close_last || slot_of(n_steps - 1) >= 0);
    if (pending && (need || close_last)) {
        TRY(launch_head(sys, W, mode, lab, true, true, 0, n_steps - 1, n_steps > 0 ? slot_of(n_steps - 1) : -1, cv,
                        eps, en, T, 0, st));
        pending = false;
    }
    return RID_OK;
}

// Run a pending closing half-step (no trace) so that f, v are complete.
static int settle(rid_system* sys, cudaStream_t st) {
    if (!sys->pending) return RID_OK;
    TRY(launch_head(sys, sys->W_act, sys->has_ens ? 1 : 0, nullptr, true, true, 0, -1, -1, nullptr, nullptr, nullptr,
                    0, 0, st));
    sys->pending = false;
    return RID_OK;
}

// --- resident walker session ------------------------------------------------
static int do_load(rid_system* sys, int W, const float* x0, const float* v0, uint64_t step0, int mem, cudaStream_t st) {
    if (W < 1) return fail(RID_ERR_ARG, "n_walkers=%d must be >= 1", W);
    if (!x0) return fail(RID_ERR_ARG, "NULL x0");
    if (mem != RID_MEM_HOST && mem != RID_MEM_DEVICE) return fail(RID_ERR_ARG, "mem must be RID_MEM_HOST or RID_MEM_DEVICE");
    if (step0 > (1ull << 32)) return fail(RID_ERR_ARG, "step0 exceeds 2^32");
    if ((long long)W * sys->S.N > (1ll << 31)) return fail(RID_ERR_ARG, "n_walkers * n_beads too large");
    TRY(check_device(sys));
    TRY(ensure_state(sys, W));
    const long long nb = (long long)W * sys->S.N;
    StateDev sd = state_view(sys);
    TRY(load_xyz(sys, x0, sd.x, nb, mem, st));
    ++sys->launches;
    if (v0) { TRY(load_xyz(sys, v0, sd.v, nb, mem, st)); ++sys->launches; }
    else { rid_launch_mb(sys->S, sd, W, (uint32_t)step0, st); ++sys->launches; }
    CK(cudaMemsetAsync(sys->flags.p, 0, (size_t)W * sizeof(int), st));
    TRY(evaluate_at_rest(sys, W, sys->has_ens ? 1 : 0, nullptr, st));
    sys->pending = false;
    sys->W_act = W;
    sys->step_next = step0;
    sys->loaded = true;
    return RID_OK;
}

// Steps of resident walkers from step_next on, traces into cv / eps / en
// ([W][T][...] device).  A run of at least two chunks (a chunk: the multiple
// of output_freq nearest 256 steps) without an energy trace is replayed as a
// CUDA graph of one chunk: the integrator then reads its Philox step from a
// device base that the graph advances, each chunk ends with the closing half
// of its last step (its last step has a trace slot), and the chunk's traces go
// from a staging block to their slots.  The arithmetic is that of the direct
// run, so the results are the same bits; only the launches are fewer.
// Whether an exploration call runs in one persistent launch (k_explore_small):
// FP32 ensembles of a shape whose walker, ensemble and CVs fit one CTA's shared
// memory, walkers in one wave, no energy trace, profiling off.
static bool fused_explore(const rid_system* sys, int W, int mode, const double* en) {
    if (!sys->fused_on || mode != 1 || sys->precision != RID_PREC_FP32 || en || sys->prof_on) return false;
    static int nsm[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    int& n = nsm[dev & 63];
    if (n == 0 && cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
    return W <= n && rid_explore_small_smem(sys->S, sys->E) > 0;
}

static int advance_steps(rid_system* sys, int W, int mode, int64_t n_steps, float* cv, float* eps, double* en,
                         long long T, cudaStream_t st) {
    const int of = sys->S.output_freq, C = sys->S.C;
    const long long chunk = std::max<long long>(of, ((256 + of - 1) / of) * of);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cs));
    if (n_steps > 0 && fused_explore(sys, W, mode, en)) {
        // every step in one launch: the same arithmetic as the per-step kernels, and the
        // call ends with its last step closed (as a settled per-step call)
        TRY(settle(sys, st));
        StateDev sd = state_view(sys);
        sd.W = W;
        cudaError_t le = cudaSuccess;
        TRY(timed_launch(sys, "k_explore_small", st, [&] {
            le = rid_launch_explore_small(sys->S, sd, sys->E, W, n_steps, (uint32_t)sys->step_next, cv, eps, T, st);
        }));
        if (le != cudaSuccess) return fail(RID_ERR_CUDA, "k_explore_small launch: %s", cudaGetErrorString(le));
        sys->pending = false;
        return RID_OK;
    }
    if (n_steps < 2 * chunk || en || sys->prof_on || cs != cudaStreamCaptureStatusNone)
        return run_steps(sys, W, mode, nullptr, n_steps, sys->step_next, cv, eps, en, T, sys->pending, false, st);
    TRY(ensure_side(sys));
    TRY(settle(sys, st));
    const long long tc = chunk / of, nchunk = n_steps / chunk;
    TRY(sys->d_stepbase.ensure(sizeof(uint32_t)));
    TRY(sys->tr_chunk.ensure((size_t)W * tc * (C + 1) * sizeof(float)));
    float* ccv = sys->tr_chunk.as<float>();
    float* ceps = ccv + (size_t)W * tc * C;
    CK(cudaMemsetAsync(sys->d_stepbase.p, 0, sizeof(uint32_t), st));
    rid_launch_add_u32(sys->d_stepbase.as<uint32_t>(), (uint32_t)sys->step_next, st);
    // capture one chunk on a private stream (the caller's may be the legacy
    // default stream, which cannot be captured; nothing runs during a capture)
    if (!sys->cap_stream) CK(cudaStreamCreateWithFlags(&sys->cap_stream, cudaStreamNonBlocking));
    cudaStream_t cst = sys->cap_stream;
    const long long l0 = sys->launches;
    CK(cudaStreamBeginCapture(cst, cudaStreamCaptureModeRelaxed));
    sys->graph_mode = true;
    bool pend = false;
    int rc = run_steps(sys, W, mode, nullptr, chunk, 0, cv ? ccv : nullptr, eps ? ceps : nullptr, nullptr, tc, pend,
                       false, cst);
    if (rc == RID_OK) rid_launch_add_u32(sys->d_stepbase.as<uint32_t>(), (uint32_t)chunk, cst);
    sys->graph_mode = false;
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cst, &g);
    if (rc != RID_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (ec != cudaSuccess) return fail(RID_ERR_CUDA, "stream capture: %s", cudaGetErrorString(ec));
    cudaGraphExec_t ge = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return fail(RID_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ei));
    // the capture counted one chunk's kernels; every replay launches them again
    sys->launches += (nchunk - 1) * (sys->launches - l0);
    cudaError_t e = cudaSuccess;
    for (long long k = 0; k < nchunk && e == cudaSuccess; ++k) {
        e = cudaGraphLaunch(ge, st);
        if (e == cudaSuccess && cv)
            e = cudaMemcpy2DAsync(cv + (size_t)k * tc * C, (size_t)T * C * sizeof(float), ccv,
                                  (size_t)tc * C * sizeof(float), (size_t)tc * C * sizeof(float), W,
                                  cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && eps)
            e = cudaMemcpy2DAsync(eps + (size_t)k * tc, (size_t)T * sizeof(float), ceps, (size_t)tc * sizeof(float),
                                  (size_t)tc * sizeof(float), W, cudaMemcpyDeviceToDevice, st);
    }
    cudaGraphExecDestroy(ge);
    if (e != cudaSuccess) return fail(RID_ERR_CUDA, "graph replay: %s", cudaGetErrorString(e));
    sys->pending = false;
    // the remainder, directly, with the Philox step read from the same device base
    const long long rem = n_steps - nchunk * chunk;
    if (rem > 0) {
        const long long tr = rem / of;
        sys->graph_mode = true;
        rc = run_steps(sys, W, mode, nullptr, rem, 0, cv ? ccv : nullptr, eps ? ceps : nullptr, nullptr, tr,
                       sys->pending, false, st);
        sys->graph_mode = false;
        TRY(rc);
        rid_launch_add_u32(sys->d_stepbase.as<uint32_t>(), (uint32_t)rem, st);
        if (tr > 0 && cv)
            CK(cudaMemcpy2DAsync(cv + (size_t)nchunk * tc * C, (size_t)T * C * sizeof(float), ccv,
                                 (size_t)tr * C * sizeof(float), (size_t)tr * C * sizeof(float), W,
                                 cudaMemcpyDeviceToDevice, st));
        if (tr > 0 && eps)
            CK(cudaMemcpy2DAsync(eps + (size_t)nchunk * tc, (size_t)T * sizeof(float), ceps, (size_t)tr * sizeof(float),
                                 (size_t)tr * sizeof(float), W, cudaMemcpyDeviceToDevice, st));
    }
    return RID_OK;
}

static int do_advance(rid_system* sys, int64_t n_steps, float* cv_out, float* eps_out, double* energy_out, int mem,
                      cudaStream_t st) {
    if (!sys->loaded) return fail(RID_ERR_STATE, "no walkers loaded");
    if (n_steps < 0) return fail(RID_ERR_ARG, "n_steps < 0");
    if (mem != RID_MEM_HOST && mem != RID_MEM_DEVICE) return fail(RID_ERR_ARG, "mem must be RID_MEM_HOST or RID_MEM_DEVICE");
    if (sys->step_next + (uint64_t)n_steps > (1ull << 32)) return fail(RID_ERR_ARG, "step counter would exceed 2^32");
    TRY(check_device(sys));
    const int W = sys->W_act, C = sys->S.C, of = sys->S.output_freq;
    (void)of;
    const long long T = n_steps / of;
    const int mode = sys->has_ens ? 1 : 0;
    float* dcv = cv_out;
    float* deps = eps_out;
    double* den = energy_out;
    if (mem == RID_MEM_HOST) {
        if (cv_out) { TRY(sys->tr_cv.ensure((size_t)W * T * C * sizeof(float))); dcv = sys->tr_cv.as<float>(); }
        if (eps_out) { TRY(sys->tr_eps.ensure((size_t)W * T * sizeof(float))); deps = sys->tr_eps.as<float>(); }
        if (energy_out) { TRY(sys->tr_en.ensure((size_t)W * T * 3 * sizeof(double))); den = sys->tr_en.as<double>(); }
    }
    TRY(advance_steps(sys, W, mode, n_steps, dcv, deps, den, T, st));
    sys->step_next += (uint64_t)n_steps;
    if (mem == RID_MEM_HOST && T > 0 && (cv_out || eps_out || energy_out)) {
        if (cv_out) CK(cudaMemcpyAsync(cv_out, dcv, (size_t)W * T * C * sizeof(float), cudaMemcpyDeviceToHost, st));
        if (eps_out) CK(cudaMemcpyAsync(eps_out, deps, (size_t)W * T * sizeof(float), cudaMemcpyDeviceToHost, st));
        if (energy_out) CK(cudaMemcpyAsync(energy_out, den, (size_t)W * T * 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return RID_OK;
}

static int do_read(rid_system* sys, float* x_out, float* v_out, uint64_t* step_next, int mem, cudaStream_t st) {
    if (!sys->loaded) return fail(RID_ERR_STATE, "no walkers loaded");
    if (mem != RID_MEM_HOST && mem != RID_MEM_DEVICE) return fail(RID_ERR_ARG, "mem must be RID_MEM_HOST or RID_MEM_DEVICE");
    TRY(check_device(sys));
    TRY(settle(sys, st));
    const int W = sys->W_act;
    const long long nb = (long long)W * sys->S.N;
    StateDev sd = state_view(sys);
    if (x_out) { TRY(store_xyz(sys, sd.x, x_out, nb, mem, st)); ++sys->launches; }
    if (v_out) { TRY(store_xyz(sys, sd.v, v_out, nb, mem, st)); ++sys->launches; }
    if (step_next) *step_next = sys->step_next;
    bool bad = false;
    TRY(fetch_flags(sys, W, st, &bad));
    if (bad) return fail(RID_ERR_NONFINITE, "non-finite force or velocity in at least one walker");
    return RID_OK;
}

// --- operations for the request loop (rid_server.cu) ------------------------
int rid_sys_load(rid_system* sys, int W, const float* x0, const float* v0, uint64_t step0, cudaStream_t st) {
    TRY(do_load(sys, W, x0, v0, step0, RID_MEM_HOST, st));
    TRY(sys->d_stepbase.ensure(sizeof(uint32_t)));
    CK(cudaMemsetAsync(sys->d_stepbase.p, 0, sizeof(uint32_t), st));
    rid_launch_add_u32(sys->d_stepbase.as<uint32_t>(), (uint32_t)step0, st);
    CK(cudaGetLastError());
    return RID_OK;
}

void rid_sys_serving(rid_system* sys, bool on) {
    sys->serving = on;
    if (!on) {   // the next direct use tunes again
        sys->ff_W = -1;
        sys->tcv.cs_W = -1;
        sys->tcv.tuned_W = -1;
    }
}

int rid_sys_graph_advance(rid_system* sys, int64_t n_steps, float* dcv, float* deps, cudaStream_t st,
                          cudaGraphExec_t* out) {
    if (!sys->loaded) return fail(RID_ERR_STATE, "no walkers loaded");
    const int of = sys->S.output_freq;
    if (n_steps < 1 || n_steps % of) return fail(RID_ERR_ARG, "graph chunk must be a positive multiple of output_freq");
    if (sys->prof_on) return fail(RID_ERR_STATE, "kernel profiling is on");
    if (!sys->d_stepbase.p) return fail(RID_ERR_STATE, "walkers were not loaded for graph replay");
    TRY(check_device(sys));
    TRY(ensure_side(sys));
    TRY(settle(sys, st));
    const int W = sys->W_act, mode = sys->has_ens ? 1 : 0;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
    sys->graph_mode = true;
    bool pend = false;
    int rc = run_steps(sys, W, mode, nullptr, n_steps, 0, dcv, deps, nullptr, n_steps / of, pend, false, st);
    if (rc == RID_OK) rid_launch_add_u32(sys->d_stepbase.as<uint32_t>(), (uint32_t)n_steps, st);
    sys->graph_mode = false;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc != RID_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(RID_ERR_CUDA, "stream capture: %s", cudaGetErrorString(e));
    const cudaError_t ei = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return fail(RID_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ei));
    sys->pending = pend;
    return RID_OK;
}

int rid_sys_advance(rid_system* sys, int64_t n_steps, float* dcv, float* deps, cudaStream_t st) {
    if (!sys->loaded) return fail(RID_ERR_STATE, "no walkers loaded");
    TRY(check_device(sys));
    const int W = sys->W_act, mode = sys->has_ens ? 1 : 0, of = sys->S.output_freq;
    TRY(ensure_side(sys));
    sys->graph_mode = true;   // Philox step = device base + t, as in the replayed graph
    const int rc = run_steps(sys, W, mode, nullptr, n_steps, 0, dcv, deps, nullptr, n_steps / of, sys->pending,
                             false, st);
    sys->graph_mode = false;
    TRY(rc);
    rid_launch_add_u32(sys->d_stepbase.as<uint32_t>(), (uint32_t)n_steps, st);
    CK(cudaGetLastError());
    return RID_OK;
}

int rid_sys_read_async(rid_system* sys, float* dx, float* dv, cudaStream_t st) {
    if (!sys->loaded) return fail(RID_ERR_STATE, "no walkers loaded");
    TRY(settle(sys, st));
    const long long nb = (long long)sys->W_act * sys->S.N;
    StateDev sd = state_view(sys);
    if (dx) rid_launch_unpack(sd.x, dx, nb, st);
    if (dv) rid_launch_unpack(sd.v, dv, nb, st);
    CK(cudaGetLastError());
    return RID_OK;
}

int rid_sys_flags(rid_system* sys, cudaStream_t st, bool* any_bad) { return fetch_flags(sys, sys->W_act, st, any_bad); }

size_t rid_sys_footprint(const rid_system* sys, int W) {
    const size_t N = sys->S.N, C = sys->S.C, nb = (size_t)W * N, nc = (size_t)W * C;
    size_t b = 4 * 16 * nb + nc * (4 + 64 + 8) + (size_t)W * (4 + 8 + 4) + 2 * 12 * nb;
    if (sys->has_ens) {
        const EnsDev& E = sys->E;
        b += (size_t)E.M * nc * 4 + (size_t)E.M * W * 4;
        if (sys->precision == RID_PREC_FP32) b += rid_mlp_fp32_scratch_floats(W, E.M, E.L, E.H) * 4;
        else b += (size_t)E.M * ((W + 127) / 128) * 128 * (E.H * (E.L * 2 + (E.resnet ? 4 : 0)) + TC_MAX_QSLICES * 4);
    }
    return b;
}

extern "C" int rid_walkers_load(rid_system* sys, int32_t W, const float* x0, const float* v0, uint64_t step0,
                                int32_t mem, void* stream) {
    if (!sys) return fail(RID_ERR_ARG, "NULL system");
    cudaStream_t st = (cudaStream_t)stream;
    TRY(do_load(sys, W, x0, v0, step0, mem, st));
    CK(cudaStreamSynchronize(st));
    return RID_OK;
}

extern "C" int rid_walkers_advance(rid_system* sys, int64_t n_steps, float* cv_out, float* eps_out,
                                   double* energy_out, int32_t mem, void* stream) {
    NvtxScope nvtx_("rid_walkers_advance");
    if (!sys) return fail(RID_ERR_ARG, "NULL system");
    return do_advance(sys, n_steps, cv_out, eps_out, energy_out, mem, (cudaStream_t)stream);
}

extern "C" int rid_walkers_read(rid_system* sys, float* x_out, float* v_out, uint64_t* step_next, int32_t mem,
                                void* stream) {
    if (!sys) return fail(RID_ERR_ARG, "NULL system");
    return do_read(sys, x_out, v_out, step_next, mem, (cudaStream_t)stream);
}

extern "C" int rid_profile_enable(rid_system* sys, int32_t enable) {
    if (!sys) return fail(RID_ERR_ARG, "NULL system");
    for (auto& r : sys->prof_recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    sys->prof_recs.clear();
    sys->prof_names.clear();
    sys->prof_on = enable != 0;
    return RID_OK;
}

extern "C" int rid_profile_read(rid_system* sys, int32_t max_kernels, char* names_out, double* total_ms,
                                int64_t* launches, int32_t* n_kernels) {
    if (!sys || max_kernels < 0 || (max_kernels > 0 && (!names_out || !total_ms || !launches)))
        return fail(RID_ERR_ARG, "bad arguments");
    const int K = (int)sys->prof_names.size();
    std::vector<double> ms(K, 0.0);
    std::vector<long long> cnt(K, 0);
    for (auto& r : sys->prof_recs) {
        CK(cudaEventSynchronize(r.b));
        float e = 0.f;
        CK(cudaEventElapsedTime(&e, r.a, r.b));
        ms[r.id] += e;
        cnt[r.id] += 1;
    }
    for (int k = 0; k < K && k < max_kernels; ++k) {
        std::snprintf(names_out + 48 * k, 48, "%s", sys->prof_names[k].c_str());
        total_ms[k] = ms[k];
        launches[k] = cnt[k];
    }
    if (n_kernels) *n_kernels = K;
    return RID_OK;
}

extern "C" int64_t rid_launch_count(rid_system* sys) { return sys ? sys->launches : -1; }

extern "C" int rid_set_mlp_cluster(rid_system* sys, int32_t csize) {
    if (!sys) return fail(RID_ERR_ARG, "NULL system");
    if (csize != 0 && csize != 1 && csize != 2 && csize != 4)
        return fail(RID_ERR_ARG, "cluster size %d: expected 0 (tuned), 1, 2 or 4", csize);
    sys->cs_force = csize;
    return RID_OK;
}

extern "C" int rid_set_ff_threads(rid_system* sys, int32_t threads) {
    if (!sys) return fail(RID_ERR_ARG, "NULL system");
    const int dth = rid_ff_default_threads(sys->S.N);
    if (threads != 0 && (threads < 32 || threads > dth || threads % 32))
        return fail(RID_ERR_ARG, "force-field CTA size %d: expected 0 (tuned) or a multiple of 32 in [32, %d]", threads,
                    dth);
    sys->ff_force = threads;
    sys->ff_W = -1;
    return RID_OK;
}

extern "C" int rid_get_ff_threads(rid_system* sys, int32_t* threads) {
    if (!sys || !threads) return fail(RID_ERR_ARG, "NULL argument");
    *threads = sys->ff_force ? sys->ff_force : (sys->ff_W >= 0 ? sys->ff_th : rid_ff_default_threads(sys->S.N));
    return RID_OK;
}

extern "C" int rid_set_fused_steps(rid_system* sys, int32_t on) {
    if (!sys) return fail(RID_ERR_ARG, "NULL system");
    if (on != 0 && on != 1) return fail(RID_ERR_ARG, "fused steps: expected 0 or 1, got %d", on);
    sys->fused_on = on != 0;
    return RID_OK;
}

extern "C" int rid_get_mlp_cluster(rid_system* sys, int32_t* csize) {
    if (!sys || !csize) return fail(RID_ERR_ARG, "NULL argument");
    *csize = sys->has_ens && sys->precision != RID_PREC_FP32 ? sys->tcv.used_cs : 0;
    return RID_OK;
}

extern "C" int rid_explore(rid_system* sys, int32_t W, const float* x0, const float* v0, uint64_t step0,
                           int64_t n_steps, float* cv_out, float* eps_out, double* energy_out, float* x_out,
                           float* v_out, int32_t mem, void* stream) {
    NvtxScope nvtx_("rid_explore");
    if (!sys || !x0) return fail(RID_ERR_ARG, "NULL argument");
    if (n_steps < 0) return fail(RID_ERR_ARG, "n_steps < 0");
    if (step0 + (uint64_t)n_steps > (1ull << 32)) return fail(RID_ERR_ARG, "step0 + n_steps exceeds 2^32");
    cudaStream_t st = (cudaStream_t)stream;
    TRY(do_load(sys, W, x0, v0, step0, mem, st));
    TRY(do_advance(sys, n_steps, cv_out, eps_out, energy_out, mem, st));
    return do_read(sys, x_out, v_out, nullptr, mem, st);
}

extern "C" int rid_label(rid_system* sys, int32_t R, const float* x0, const float* v0, const double* s0,
                         const double* kappa, uint64_t step0, int64_t n_steps, int64_t n_equil, int32_t n_blocks,
                         double* mf_out, double* se_out, double* std_out, float* x_out, float* v_out, int32_t mem,
                         void* stream) {
    NvtxScope nvtx_("rid_label");
    if (!sys || !x0 || !s0 || !kappa || !mf_out || !se_out || !std_out) return fail(RID_ERR_ARG, "NULL argument");
    if (R < 1) return fail(RID_ERR_ARG, "n_runs=%d must be >= 1", R);
    if (mem != RID_MEM_HOST && mem != RID_MEM_DEVICE) return fail(RID_ERR_ARG, "mem must be RID_MEM_HOST or RID_MEM_DEVICE");
    if (n_blocks < 2 || n_blocks > RID_MAX_BLOCKS) return fail(RID_ERR_ARG, "n_blocks=%d outside [2, %d]", n_blocks, RID_MAX_BLOCKS);
    if (n_equil < 0 || n_steps - n_equil < n_blocks) return fail(RID_ERR_ARG, "need 0 <= n_equil and n_steps - n_equil >= n_blocks");
    if (step0 + (uint64_t)n_steps > (1ull << 32)) return fail(RID_ERR_ARG, "step0 + n_steps exceeds 2^32");
    TRY(check_device(sys));
    sys->loaded = false;   // these calls reuse the resident walker buffers
    sys->pending = false;
    cudaStream_t st = (cudaStream_t)stream;
    TRY(ensure_state(sys, R));
    const int N = sys->S.N, C = sys->S.C;
    const long long nb = (long long)R * N, nc = (long long)R * C;
    TRY(sys->lsum.ensure(nc * sizeof(double)));
    TRY(sys->lsum2.ensure(nc * sizeof(double)));
    TRY(sys->lbsum.ensure(nc * n_blocks * sizeof(double)));
    TRY(sys->ls0.ensure(nc * sizeof(double)));
    TRY(sys->lkap.ensure(nc * sizeof(double)));
    const cudaMemcpyKind k = mem == RID_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    CK(cudaMemcpyAsync(sys->ls0.p, s0, nc * sizeof(double), k, st));
    CK(cudaMemcpyAsync(sys->lkap.p, kappa, nc * sizeof(double), k, st));
    CK(cudaMemsetAsync(sys->lsum.p, 0, nc * sizeof(double), st));
    CK(cudaMemsetAsync(sys->lsum2.p, 0, nc * sizeof(double), st));
    CK(cudaMemsetAsync(sys->lbsum.p, 0, nc * n_blocks * sizeof(double), st));
    LabelDev lab{};
    lab.s0 = sys->ls0.as<double>();
    lab.kappa = sys->lkap.as<double>();
    lab.sum = sys->lsum.as<double>();
    lab.sum2 = sys->lsum2.as<double>();
    lab.bsum = sys->lbsum.as<double>();
    lab.B = n_blocks;
    lab.n_equil = n_equil;
    lab.K = n_steps - n_equil;
    StateDev sd = state_view(sys);
    TRY(load_xyz(sys, x0, sd.x, nb, mem, st));
    if (v0) TRY(load_xyz(sys, v0, sd.v, nb, mem, st));
    CK(cudaMemsetAsync(sys->flags.p, 0, (size_t)R * sizeof(int), st));
    double *dmf = mf_out, *dse = se_out, *dsd = std_out;
    if (mem == RID_MEM_HOST) {
        TRY(sys->out_mf.ensure(nc * sizeof(double)));
        TRY(sys->out_se.ensure(nc * sizeof(double)));
        TRY(sys->out_sd.ensure(nc * sizeof(double)));
        dmf = sys->out_mf.as<double>();
        dse = sys->out_se.as<double>();
        dsd = sys->out_sd.as<double>();
    }
    if (sys->fused_on && N < 768 && !sys->prof_on) {
        // chains below 768 beads: every step of every run in one launch of the persistent
        // label kernel, one CTA per run (the batch and the request loop's kernel: the same
        // arithmetic as the per-step kernels, so the same bits)
        FusedJob J{};
        J.S = sys->S;
        J.x = sd.x;
        J.v = sd.v;
        J.f = sd.f;
        J.s0 = lab.s0;
        J.kappa = lab.kappa;
        J.sum = lab.sum;
        J.sum2 = lab.sum2;
        J.bsum = lab.bsum;
        J.mf = dmf;
        J.se = dse;
        J.sd = dsd;
        J.flags = sd.flags;
        J.R = R;
        J.B = n_blocks;
        J.n_steps = n_steps;
        J.n_equil = n_equil;
        J.K = n_steps - n_equil;
        J.t0 = 0;
        J.t1 = n_steps;
        J.step0 = (uint32_t)step0;
        J.init = 1;
        J.mb = v0 ? 0 : 1;
        std::vector<FusedItem> items((size_t)R);
        for (int r = 0; r < R; ++r) items[r] = {0, r};
        const size_t o_items = (sizeof(FusedJob) + 255) / 256 * 256;
        const size_t o_cnt = (o_items + sizeof(FusedItem) * (size_t)R + 255) / 256 * 256;
        TRY(sys->lfused.ensure(o_cnt + 256));
        std::vector<char> hb(o_cnt);
        memcpy(hb.data(), &J, sizeof(FusedJob));
        memcpy(hb.data() + o_items, items.data(), sizeof(FusedItem) * (size_t)R);
        char* dm = sys->lfused.as<char>();
        CK(cudaMemcpyAsync(dm, hb.data(), o_cnt, cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(dm + o_cnt, 0, 256, st));
        FusedArgs A{};
        A.jobs = reinterpret_cast<const FusedJob*>(dm);
        A.items = reinterpret_cast<const FusedItem*>(dm + o_items);
        A.n_items = R;
        A.next = reinterpret_cast<int*>(dm + o_cnt);
        const size_t smem = rid_label_fused_smem(N, C, 0);
        int nt = N <= 128 ? 128 : (N <= 256 ? 256 : 512);
        if (rid_label_fused_occupancy(nt, smem) < 1) nt = 128;
        int occ = rid_label_fused_occupancy(nt, smem);
        if (occ < 1) return fail(RID_ERR_ARG, "label runs of %d beads exceed shared memory", N);
        int nsm = 1, dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        const int grid = (int)std::min<long long>(R, (long long)occ * nsm);
        cudaError_t le = cudaSuccess;
        TRY(timed_launch(sys, "k_label_fused", st, [&] { le = rid_launch_label_fused(A, nt, grid, smem, st); }));
        if (le != cudaSuccess) return fail(RID_ERR_CUDA, "k_label_fused launch: %s", cudaGetErrorString(le));
        // the host staging vector must outlive the copy
        CK(cudaStreamSynchronize(st));
    } else {
        if (!v0) rid_launch_mb(sys->S, sd, R, (uint32_t)step0, st);
        TRY(evaluate_at_rest(sys, R, 2, &lab, st));
        bool pend = false;
        TRY(run_steps(sys, R, 2, &lab, n_steps, step0, nullptr, nullptr, nullptr, 0, pend, true, st));
        rid_launch_label_final(lab, R, C, dmf, dse, dsd, st);
    }
    CK(cudaGetLastError());
    TRY(store_xyz(sys, sd.x, x_out, nb, mem, st));
    TRY(store_xyz(sys, sd.v, v_out, nb, mem, st));
    if (mem == RID_MEM_HOST) {
        CK(cudaMemcpyAsync(mf_out, dmf, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(se_out, dse, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(std_out, dsd, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    bool bad = false;
    TRY(fetch_flags(sys, R, st, &bad));
    if (bad) return fail(RID_ERR_NONFINITE, "non-finite force or velocity in at least one run");
    return RID_OK;
}

// MCMC dimension reduction with the system's own ensemble evaluation
// (k_mcmc.cu kernels around launch_mlp): proposals are written as the MLP
// input of W resident walkers and the member values come from the ensemble
// kernels at the precision the ensemble was set with.  The walker buffers are
// reused (like rid_label); scratch for the chain state and histograms is
// allocated for the call.
extern "C" int rid_mcmc_system(rid_system* sys, int32_t W, const float* s0, int64_t n_steps, int64_t n_burn,
                               double kT, double step_size, uint64_t seed, int32_t bins, int32_t proj_i,
                               int32_t proj_j, const double* cv_lo, const double* cv_hi, const rid_mcmc_path* path,
                               float* s_out, uint64_t* hist1_out,
                               uint64_t* hist2_out, double* pmf1_out, double* pmf2_out, uint64_t* histp_out,
                               double* pmfp_out, int64_t* n_accepted, int32_t mem, void* stream) {
    NvtxScope nvtx_("rid_mcmc_system");
    if (!sys || !s0) return fail(RID_ERR_ARG, "NULL argument");
    if (mem != RID_MEM_HOST && mem != RID_MEM_DEVICE) return fail(RID_ERR_ARG, "mem must be RID_MEM_HOST or RID_MEM_DEVICE");
    if (!sys->has_ens) return fail(RID_ERR_STATE, "no ensemble set");
    const int C = sys->S.C;
    if (W < 1 || n_steps < 0 || n_steps > 0xFFFFFFFFll || n_burn < 0 || !(kT > 0) || !(step_size >= 0) || bins < 1 ||
        bins > 4096 || proj_i < 0 || proj_i >= C || proj_j < 0 || proj_j >= C)
        return fail(RID_ERR_ARG, "mcmc: parameters out of range");
    if ((long long)W * sys->S.N > (1ll << 31)) return fail(RID_ERR_ARG, "n_walkers * n_beads too large");
    const int NP = path ? path->n_nodes : 0, Cp = path ? path->n_cv : 0;
    if (path) TRY(rid_mc_path_check(NP, Cp, C, path->cv, path->nodes, path->lambda, path->z_lo, path->z_hi));
    std::vector<int32_t> kinds(C, 0);
    if (sys->has_dist) {
        CK(cudaMemcpy(kinds.data(), sys->d_cvdist.p, sizeof(int) * C, cudaMemcpyDeviceToHost));
        TRY(rid_mc_range_check(C, kinds.data(), cv_lo, cv_hi));
    }
    TRY(check_device(sys));
    sys->loaded = false;   // the resident walker buffers are reused
    sys->pending = false;
    cudaStream_t st = (cudaStream_t)stream;
    TRY(ensure_state(sys, W));
    StateDev sd = state_view(sys);
    sd.W = W;
    const long long nS = (long long)W * C, n1 = (long long)C * bins, n2 = (long long)bins * bins;
    struct Scoped {
        DevBuf b;
        ~Scoped() { b.release(); }
    } scoped;
    // counters first (zeroed together), then the PMFs, states and path nodes
    const long long np2 = NP ? n2 : 0, npn = (long long)NP * Cp;
    const size_t o_h1 = 0, o_h2 = o_h1 + 8 * n1, o_hp = o_h2 + 8 * n2, o_na = o_hp + 8 * np2, o_p1 = o_na + 16;
    const size_t o_p2 = o_p1 + 8 * n1, o_pp = o_p2 + 8 * n2, o_s = o_pp + 8 * np2, o_sp = o_s + 4 * nS;
    const size_t o_A = o_sp + 4 * nS, o_pn = o_A + ((4 * (size_t)W + 15) & ~(size_t)15), o_pc = o_pn + 4 * npn;
    const size_t o_rg = o_pc + 4 * (size_t)Cp;   // distance-CV ranges lo [C], hi [C]
    TRY(scoped.b.ensure(o_rg + 8 * (size_t)C));
    unsigned char* b = static_cast<unsigned char*>(scoped.b.p);
    auto* h1 = reinterpret_cast<unsigned long long*>(b + o_h1);
    auto* h2 = reinterpret_cast<unsigned long long*>(b + o_h2);
    auto* na = reinterpret_cast<unsigned long long*>(b + o_na);
    double* p1 = reinterpret_cast<double*>(b + o_p1);
    double* p2 = reinterpret_cast<double*>(b + o_p2);
    float* ds = reinterpret_cast<float*>(b + o_s);
    float* dsp = reinterpret_cast<float*>(b + o_sp);
    float* dA = reinterpret_cast<float*>(b + o_A);
    double* pp = reinterpret_cast<double*>(b + o_pp);
    McPathDev pd;
    if (NP) {
        pd.n_nodes = NP;
        pd.n_cv = Cp;
        pd.nodes = reinterpret_cast<float*>(b + o_pn);
        pd.cv = reinterpret_cast<int*>(b + o_pc);
        pd.lambda = (float)path->lambda;
        pd.z_lo = (float)path->z_lo;
        pd.z_hi = (float)path->z_hi;
        pd.hist = reinterpret_cast<unsigned long long*>(b + o_hp);
        CK(cudaMemcpyAsync(b + o_pn, path->nodes, 4 * npn, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(b + o_pc, path->cv, 4 * (size_t)Cp, cudaMemcpyHostToDevice, st));
    }
    const cudaMemcpyKind kin = mem == RID_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind kout = mem == RID_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    McCvDev cvk;
    std::vector<float> rg(2 * (size_t)C, 0.0f);
    if (sys->has_dist) {
        for (int c = 0; c < C; ++c)
            if (kinds[c]) {
                rg[c] = (float)cv_lo[c];
                rg[C + c] = (float)cv_hi[c];
            }
        CK(cudaMemcpy(b + o_rg, rg.data(), 8 * (size_t)C, cudaMemcpyHostToDevice));
        cvk.dist = sys->d_cvdist.as<int>();
        cvk.lo = reinterpret_cast<float*>(b + o_rg);
        cvk.hi = cvk.lo + C;
    }
    CK(cudaMemcpyAsync(ds, s0, sizeof(float) * nS, kin, st));
    CK(cudaMemsetAsync(b, 0, o_p1, st));
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const int M = sys->E.M, nav = M * sys->E.aslices;
    rid_launch_mc_features(ds, sd.u, nS, C, cvk, st);
    TRY(launch_mlp(sys, W, 1, sd, st, true));
    rid_launch_mc_accept_values(sd.Aval, nav, M, W, C, ds, dsp, dA, 0u, (float)kT, k0, k1, 1, 0, bins, proj_i, proj_j,
                                h1, h2, na, pd, cvk, st);
    for (int64_t t = 0; t < n_steps; ++t) {
        rid_launch_mc_propose(ds, dsp, sd.u, W, C, (uint32_t)t, (float)step_size, k0, k1, cvk, st);
        TRY(launch_mlp(sys, W, 1, sd, st, true));
        rid_launch_mc_accept_values(sd.Aval, nav, M, W, C, ds, dsp, dA, (uint32_t)t, (float)kT, k0, k1, 0,
                                    t >= n_burn, bins, proj_i, proj_j, h1, h2, na, pd, cvk, st);
    }
    rid_launch_mc_pmf(h1, C, bins, kT, p1, st);
    rid_launch_mc_pmf(h2, 1, (int)n2, kT, p2, st);
    if (NP) rid_launch_mc_pmf(pd.hist, 1, (int)n2, kT, pp, st);
    CK(cudaGetLastError());
    if (s_out) CK(cudaMemcpyAsync(s_out, ds, sizeof(float) * nS, kout, st));
    if (hist1_out) CK(cudaMemcpyAsync(hist1_out, h1, 8 * n1, kout, st));
    if (hist2_out) CK(cudaMemcpyAsync(hist2_out, h2, 8 * n2, kout, st));
    if (pmf1_out) CK(cudaMemcpyAsync(pmf1_out, p1, 8 * n1, kout, st));
    if (pmf2_out) CK(cudaMemcpyAsync(pmf2_out, p2, 8 * n2, kout, st));
    if (NP && histp_out) CK(cudaMemcpyAsync(histp_out, pd.hist, 8 * n2, kout, st));
    if (NP && pmfp_out) CK(cudaMemcpyAsync(pmfp_out, pp, 8 * n2, kout, st));
    unsigned long long hna = 0;
    CK(cudaMemcpyAsync(&hna, na, sizeof(hna), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (n_accepted) *n_accepted = (int64_t)hna;
    sys->launches += 3 + 3 * n_steps + 2 + (NP ? 1 : 0);
    return RID_OK;
}

// Constrained-MD labels on distance CVs (k_label_cons.cu).  Scratch for the
// call is allocated here and released before returning.
extern "C" int rid_label_constrained(rid_system* sys, int32_t R, const float* x0, const float* v0, int32_t C,
                                     const int32_t* pairs, const double* d0, uint64_t step0, int64_t n_steps,
                                     int64_t n_equil, int32_t n_blocks, double* mf_out, double* se_out,
                                     double* std_out, float* x_out, float* v_out, int32_t mem, void* stream) {
    NvtxScope nvtx_("rid_label_constrained");
    if (!sys || !x0 || !pairs || !d0 || !mf_out || !se_out || !std_out) return fail(RID_ERR_ARG, "NULL argument");
    if (R < 1 || C < 1 || C > RID_MAX_CV) return fail(RID_ERR_ARG, "n_runs >= 1 and 1 <= n_cv <= %d required", RID_MAX_CV);
    if (mem != RID_MEM_HOST && mem != RID_MEM_DEVICE) return fail(RID_ERR_ARG, "mem must be RID_MEM_HOST or RID_MEM_DEVICE");
    if (n_blocks < 2 || n_blocks > RID_MAX_BLOCKS) return fail(RID_ERR_ARG, "n_blocks=%d outside [2, %d]", n_blocks, RID_MAX_BLOCKS);
    if (n_equil < 0 || n_steps - n_equil < n_blocks) return fail(RID_ERR_ARG, "need 0 <= n_equil and n_steps - n_equil >= n_blocks");
    if (step0 + (uint64_t)n_steps > (1ull << 32)) return fail(RID_ERR_ARG, "step0 + n_steps exceeds 2^32");
    TRY(check_device(sys));
    const int N = sys->S.N;
    std::vector<int> used(N, 0);
    std::vector<int2> hp(C);
    for (int j = 0; j < C; ++j) {
        const int a = pairs[2 * j], b = pairs[2 * j + 1];
        if (a < 0 || b < 0 || a >= N || b >= N || a == b) return fail(RID_ERR_ARG, "pair %d: beads out of range or equal", j);
        if (used[a]++ || used[b]++) return fail(RID_ERR_ARG, "pair %d shares a bead with another pair", j);
        hp[j] = make_int2(a, b);
    }
    const size_t smem = rid_label_cons_smem(N, C);
    if (smem > 227 * 1024) return fail(RID_ERR_ARG, "chain of %d beads with %d CVs exceeds shared memory", N, C);
    cudaStream_t st = (cudaStream_t)stream;
    const long long nb = (long long)R * N, nc = (long long)R * C;
    const cudaMemcpyKind kin = mem == RID_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    // host d0 (double) -> device float; x0, v0 -> float4
    std::vector<double> hd0;
    const double* d0h = d0;
    if (mem == RID_MEM_DEVICE) {
        hd0.resize(nc);
        CK(cudaMemcpyAsync(hd0.data(), d0, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        d0h = hd0.data();
    }
    std::vector<float> fd0(nc);
    for (long long i = 0; i < nc; ++i) {
        if (!(d0h[i] > 0)) return fail(RID_ERR_ARG, "d0 must be positive");
        fd0[i] = (float)d0h[i];
    }
    struct Scoped {   // released on every return (cudaFree waits for the device)
        DevBuf b;
        ~Scoped() { b.release(); }
    } scoped;
    DevBuf& buf = scoped.b;
    const size_t o_x = 0, o_v = o_x + 16 * nb, o_xo = o_v + 16 * nb, o_vo = o_xo + 16 * nb, o_io = o_vo + 16 * nb;
    const size_t o_bs = o_io + 12 * nb, o_mf = o_bs + 8 * nc * n_blocks, o_se = o_mf + 8 * nc, o_sd = o_se + 8 * nc;
    const size_t o_d0 = o_sd + 8 * nc, o_pr = o_d0 + ((4 * nc + 15) & ~15ll), o_bad = o_pr + ((8 * C + 15) & ~15);
    TRY(buf.ensure(o_bad + 4 * R));
    unsigned char* b = static_cast<unsigned char*>(buf.p);
    float4* dx = reinterpret_cast<float4*>(b + o_x);
    float4* dv = reinterpret_cast<float4*>(b + o_v);
    float4* dxo = reinterpret_cast<float4*>(b + o_xo);
    float4* dvo = reinterpret_cast<float4*>(b + o_vo);
    float* io = reinterpret_cast<float*>(b + o_io);
    double* bs = reinterpret_cast<double*>(b + o_bs);
    double* dmf = reinterpret_cast<double*>(b + o_mf);
    double* dse = reinterpret_cast<double*>(b + o_se);
    double* dsd = reinterpret_cast<double*>(b + o_sd);
    float* dd0 = reinterpret_cast<float*>(b + o_d0);
    int2* dpr = reinterpret_cast<int2*>(b + o_pr);
    int* dbad = reinterpret_cast<int*>(b + o_bad);
    CK(cudaMemcpyAsync(io, x0, (size_t)nb * 12, kin, st));
    rid_launch_pack(io, dx, nb, st);
    if (v0) {
        CK(cudaMemcpyAsync(io, v0, (size_t)nb * 12, kin, st));
        rid_launch_pack(io, dv, nb, st);
    }
    CK(cudaMemcpyAsync(dd0, fd0.data(), nc * sizeof(float), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dpr, hp.data(), C * sizeof(int2), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(bs, 0, 8 * nc * n_blocks, st));
    CK(rid_launch_label_cons(sys->S, R, C, n_blocks, n_steps, n_equil, (uint32_t)step0, (float)sys->desc.kT, dx,
                             v0 ? dv : nullptr, dpr, dd0, bs, dmf, dse, dsd, dxo, dvo, dbad, st));
    const cudaMemcpyKind kout = mem == RID_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    CK(cudaMemcpyAsync(mf_out, dmf, nc * sizeof(double), kout, st));
    CK(cudaMemcpyAsync(se_out, dse, nc * sizeof(double), kout, st));
    CK(cudaMemcpyAsync(std_out, dsd, nc * sizeof(double), kout, st));
    if (x_out) {
        rid_launch_unpack(dxo, io, nb, st);
        CK(cudaMemcpyAsync(x_out, io, (size_t)nb * 12, kout, st));
    }
    if (v_out) {
        float* io2 = reinterpret_cast<float*>(b + o_x);   // x0 staging is free by now
        rid_launch_unpack(dvo, io2, nb, st);
        CK(cudaMemcpyAsync(v_out, io2, (size_t)nb * 12, kout, st));
    }
    std::vector<int> hbad(R);
    CK(cudaMemcpyAsync(hbad.data(), dbad, R * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    ++sys->launches;
    for (int r = 0; r < R; ++r)
        if (hbad[r]) return fail(RID_ERR_NONFINITE, "non-finite force or position in run %d", r);
    return RID_OK;
}

extern "C" int rid_eval_forces(rid_system* sys, int32_t W, const float* x, int32_t bias, const double* s0,
                               const double* kappa, float* f_out, float* s_out, float* eps_out, float* abar_out,
                               float* grad_out, int32_t mem, void* stream) {
    NvtxScope nvtx_("rid_eval_forces");
    if (!sys || !x) return fail(RID_ERR_ARG, "NULL argument");
    if (W < 1) return fail(RID_ERR_ARG, "n_walkers must be >= 1");
    if (mem != RID_MEM_HOST && mem != RID_MEM_DEVICE) return fail(RID_ERR_ARG, "bad mem");
    if (bias < 0 || bias > 2) return fail(RID_ERR_ARG, "bias must be RID_BIAS_*");
    if (bias == RID_BIAS_ENSEMBLE && !sys->has_ens) return fail(RID_ERR_STATE, "no ensemble set");
    if (bias == RID_BIAS_RESTRAINT && (!s0 || !kappa)) return fail(RID_ERR_ARG, "restraint needs s0 and kappa");
    if ((eps_out || abar_out || grad_out) && bias != RID_BIAS_ENSEMBLE)
        return fail(RID_ERR_ARG, "eps/abar/grad outputs need bias = RID_BIAS_ENSEMBLE");
    TRY(check_device(sys));
    sys->loaded = false;   // these calls reuse the resident walker buffers
    sys->pending = false;
    cudaStream_t st = (cudaStream_t)stream;
    TRY(ensure_state(sys, W));
    const int N = sys->S.N, C = sys->S.C;
    const long long nb = (long long)W * N, nc = (long long)W * C;
    LabelDev lab{};
    if (bias == RID_BIAS_RESTRAINT) {
        TRY(sys->ls0.ensure(nc * sizeof(double)));
        TRY(sys->lkap.ensure(nc * sizeof(double)));
        const cudaMemcpyKind k = mem == RID_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        CK(cudaMemcpyAsync(sys->ls0.p, s0, nc * sizeof(double), k, st));
        CK(cudaMemcpyAsync(sys->lkap.p, kappa, nc * sizeof(double), k, st));
        lab.s0 = sys->ls0.as<double>();
        lab.kappa = sys->lkap.as<double>();
        lab.B = 1;
        lab.K = 1;
    }
    StateDev sd = state_view(sys);
    TRY(load_xyz(sys, x, sd.x, nb, mem, st));
    CK(cudaMemsetAsync(sys->flags.p, 0, (size_t)W * sizeof(int), st));
    TRY(evaluate_at_rest(sys, W, bias, bias == 2 ? &lab : nullptr, st));
    TRY(store_xyz(sys, sd.f, f_out, nb, mem, st));
    const cudaMemcpyKind ko = mem == RID_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (s_out) CK(cudaMemcpyAsync(s_out, sd.s, nc * sizeof(float), ko, st));
    if (eps_out) CK(cudaMemcpyAsync(eps_out, sd.eps, (size_t)W * sizeof(float), ko, st));
    if (bias == RID_BIAS_ENSEMBLE) {
        const int M = sys->E.M;
        // the per-walker rows of Aval / gradA are laid out for the call's W
        if (grad_out) CK(cudaMemcpyAsync(grad_out, sd.gradA, (size_t)M * nc * sizeof(float), ko, st));
        if (abar_out) {
            const int ns = sys->E.aslices;
            std::vector<float> a((size_t)M * ns * W);
            CK(cudaMemcpyAsync(a.data(), sd.Aval, a.size() * sizeof(float), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            std::vector<float> ab(W, 0.0f);
            for (int w = 0; w < W; ++w) {
                float acc = 0.0f;
                for (int m = 0; m < M; ++m)
                    for (int q = 0; q < ns; ++q) acc += a[((size_t)m * ns + q) * W + w];
                ab[w] = acc / (float)M;
            }
            CK(cudaMemcpyAsync(abar_out, ab.data(), W * sizeof(float),
                               mem == RID_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice, st));
        }
    }
    CK(cudaStreamSynchronize(st));
    return RID_OK;
}

extern "C" int rid_pair_mask(rid_system* sys, int32_t W, const float* x, uint32_t* mask_out, int32_t mem,
                             void* stream) {
    if (!sys || !x || !mask_out) return fail(RID_ERR_ARG, "NULL argument");
    if (W < 1) return fail(RID_ERR_ARG, "n_walkers must be >= 1");
    if (mem != RID_MEM_HOST && mem != RID_MEM_DEVICE) return fail(RID_ERR_ARG, "bad mem");
    TRY(check_device(sys));
    sys->loaded = false;   // these calls reuse the resident walker buffers
    sys->pending = false;
    cudaStream_t st = (cudaStream_t)stream;
    TRY(ensure_state(sys, W));
    const int N = sys->S.N;
    const long long nb = (long long)W * N, nw = (N + 31) / 32;
    StateDev sd = state_view(sys);
    TRY(load_xyz(sys, x, sd.x, nb, mem, st));
    uint32_t* dm = mask_out;
    if (mem == RID_MEM_HOST) {
        TRY(sys->io1.ensure((size_t)nb * nw * sizeof(uint32_t)));
        dm = sys->io1.as<uint32_t>();
    }
    rid_launch_pair_mask(sys->S, sd, W, dm, st);
    CK(cudaGetLastError());
    if (mem == RID_MEM_HOST) CK(cudaMemcpyAsync(mask_out, dm, (size_t)nb * nw * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return RID_OK;
}

extern "C" int rid_philox(int64_t n, const uint32_t* counters, uint64_t seed, uint32_t* out_words,
                          float* out_normals, int32_t mem, void* stream) {
    if (n < 0 || (n > 0 && !counters)) return fail(RID_ERR_ARG, "bad counters");
    if (mem != RID_MEM_HOST && mem != RID_MEM_DEVICE) return fail(RID_ERR_ARG, "bad mem");
    if (n == 0) return RID_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t* dc = counters;
    uint32_t* dw = out_words;
    float* dn = out_normals;
    void* tmp = nullptr;
    if (mem == RID_MEM_HOST) {
        const size_t bytes = (size_t)n * (16 + 16 + 12);
        CK(cudaMalloc(&tmp, bytes));
        char* b = (char*)tmp;
        CK(cudaMemcpyAsync(b, counters, (size_t)n * 16, cudaMemcpyHostToDevice, st));
        dc = (const uint32_t*)b;
        dw = out_words ? (uint32_t*)(b + (size_t)n * 16) : nullptr;
        dn = out_normals ? (float*)(b + (size_t)n * 32) : nullptr;
    }
    rid_launch_philox(n, dc, (uint32_t)seed, (uint32_t)(seed >> 32), dw, dn, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && mem == RID_MEM_HOST) {
        if (out_words) e = cudaMemcpyAsync(out_words, dw, (size_t)n * 16, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && out_normals) e = cudaMemcpyAsync(out_normals, dn, (size_t)n * 12, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return fail(RID_ERR_CUDA, "rid_philox: %s", cudaGetErrorString(e));
    return RID_OK;
}
