// C ABI entry points of the render path, error reporting and the device
// status word.  Argument checks happen here, on the host, before any launch.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>

#include "common.cuh"

namespace tsdfs {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local char g_msg[512] = "";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return TSDFS_OK;
    return fail(TSDFS_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// device addresses of the library's __device__ variables
//
// A __device__ variable has one instance per CUDA context, so its address is
// looked up with cudaGetSymbolAddress in the context that is current.  The
// lookup is cached per device together with the id of the context it was made
// in (cuCtxGetId: unique within the process, never reused); after a
// cudaDeviceReset the device's next context has another id, and the address is
// looked up again instead of reusing the stale one.  The two driver calls are
// reached through the runtime's driver entry point, so the library does not
// link the driver library itself.
// ---------------------------------------------------------------------------
namespace {
using CtxGetCurrentFn = int (*)(void**);
using CtxGetIdFn = int (*)(void*, unsigned long long*);
std::once_flag g_ctx_fn_once;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
}  // namespace

// id of the current context of the calling thread; 0 when there is none yet or the
// driver lacks the query (the cache then keys on the device alone)
unsigned long long current_context_id() {
    std::call_once(g_ctx_fn_once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    });
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != 0 || !ctx) return 0;
    if (g_ctx_get_id(ctx, &id) != 0) return 0;
    return id;
}

int symbol_address(SymbolCache& cache, const void* symbol, void** out, const char* what) {
    int dev = 0;
    int rc = cuda_check(cudaGetDevice(&dev), what);
    if (rc) return rc;
    if (dev < 0 || dev >= SymbolCache::kDevices) return fail(TSDFS_E_UNSUPPORTED, "%s: device index %d out of range", what, dev);
    std::lock_guard<std::mutex> lk(cache.mu);
    unsigned long long id = current_context_id();
    if (cache.addr[dev] && id != 0 && id == cache.ctx[dev]) {
        *out = cache.addr[dev];
        return TSDFS_OK;
    }
    void* p = nullptr;
    rc = cuda_check(cudaGetSymbolAddress(&p, symbol), what);
    if (rc) return rc;
    if (id == 0) id = current_context_id();   // the lookup made the device's context current
    cache.addr[dev] = p;
    cache.ctx[dev] = id;
    *out = p;
    return TSDFS_OK;
}

// test-only limits of the failure paths (tsdfs_set_test_limits)
static std::atomic<uint32_t> g_test_spin{0};
static std::atomic<int> g_test_march{0};
static std::atomic<int> g_test_withhold{-1};
uint32_t test_spin_limit(uint32_t dflt) {
    const uint32_t v = g_test_spin.load();
    return v ? v : dflt;
}
int test_march_cap() { return g_test_march.load(); }
int test_withhold_chunk() { return g_test_withhold.load(); }

// one status word per device context
static __device__ uint32_t g_status_word;
static SymbolCache g_status_cache;

uint32_t* device_status_word() {
    void* p = nullptr;
    if (symbol_address(g_status_cache, (const void*)&g_status_word, &p, "status word address")) return nullptr;
    return static_cast<uint32_t*>(p);
}

// ---------------------------------------------------------------------------
// kernel timing
// ---------------------------------------------------------------------------
struct ProfRec {
    const char* name;
    cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static ProfRec* g_prof = nullptr;
static size_t g_prof_n = 0, g_prof_cap = 0;

void prof_begin(const char* name, cudaStream_t st, void** token) {
    *token = nullptr;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return;
    if (g_prof_n == g_prof_cap) {
        size_t cap = g_prof_cap ? 2 * g_prof_cap : 1024;
        ProfRec* p = static_cast<ProfRec*>(realloc(g_prof, cap * sizeof(ProfRec)));
        if (!p) return;
        g_prof = p;
        g_prof_cap = cap;
    }
    ProfRec& r = g_prof[g_prof_n];
    if (cudaEventCreate(&r.a) != cudaSuccess) return;
    if (cudaEventCreate(&r.b) != cudaSuccess) {
        cudaEventDestroy(r.a);
        return;
    }
    r.name = name;
    cudaEventRecord(r.a, st);
    *token = reinterpret_cast<void*>(g_prof_n + 1);
    ++g_prof_n;
}

void prof_end(void* token, cudaStream_t st) {
    if (!token) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    size_t i = reinterpret_cast<size_t>(token) - 1;
    if (i < g_prof_n) cudaEventRecord(g_prof[i].b, st);
}

static void prof_clear() {
    for (size_t i = 0; i < g_prof_n; ++i) {
        cudaEventDestroy(g_prof[i].a);
        cudaEventDestroy(g_prof[i].b);
    }
    g_prof_n = 0;
}

// ---------------------------------------------------------------------------
// internal launchers (mlp_simt.cu, composite.cu, bounds.cu)
// ---------------------------------------------------------------------------
template <int ARCH>
int launch_mlp_full_simt(const NetParams& np, const SampleSource& src, SampleRec* rec, int64_t max_samples, cudaStream_t st);
template <int ARCH>
int launch_mlp_value_simt(const NetParams& np, const SampleSource& src, float* f_out, cudaStream_t st);
int launch_composite(const SampleRec* rec, const int32_t* offsets, int per_ray, const uint8_t* status, int64_t n_rays,
                     const int32_t* total_dev, int64_t capacity, Opacity op, float* rgb, float* depth,
                     float* wsum, float* normal, float* eik, cudaStream_t st);
int launch_hier_setup(const tsdfs_grid* g, const float* ray_o, const float* ray_d, int64_t n_rays, float t_near,
                      float t_far, float* t0, float* te, uint8_t* status, float* tc, float* dc, int n_c,
                      cudaStream_t st);
int launch_hier_fine(const float* fcoarse, const float* tc, const float* t0, const float* te, int64_t n_rays,
                     Opacity op, float* t_out, float* d_out, int n_c, int n_f, cudaStream_t st);
int launch_bounded_counts(const int32_t* offsets, int64_t n_rays, int n_f, int64_t max_coarse, int32_t* n2,
                          cudaStream_t st);
int launch_bounded_fine(const float* fcoarse, const int32_t* offsets, const float* t_n, const float* t_f,
                        const int32_t* offsets2, int64_t n_rays, int n_f, Opacity op, int64_t max_coarse,
                        int64_t capacity2, float* t_out, float* d_out, int32_t* ray_out, cudaStream_t st);
int grid_check(const tsdfs_grid* g);
int mlp_tc_available(int arch);
int launch_mlp_full_tc(const tsdfs_mlp* mlp, const SampleSource& src, SampleRec* rec, int64_t max_samples,
                       uint8_t* stash, cudaStream_t st);
size_t mlp_tc_stash_bytes();
int launch_mlp_value_tc(const tsdfs_mlp* mlp, const SampleSource& src, float* f_out, cudaStream_t st);
int launch_mlp_pipe(const tsdfs_mlp* mlp, const SampleSource& src, SampleRec* rec, int64_t max_samples,
                    cudaStream_t st);

// network kernel per precision (tsdfs_set_network_kernel), index = TSDFS_PREC_*
static int g_netkernel[4] = {0, TSDFS_NETKERNEL_SERIAL, TSDFS_NETKERNEL_SERIAL, TSDFS_NETKERNEL_PIPELINED};
static std::mutex g_netkernel_mu;

static int netkernel_of(int precision) {
    std::lock_guard<std::mutex> lk(g_netkernel_mu);
    return g_netkernel[precision];
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

static int mlp_check(const tsdfs_mlp* m) {
    if (!m) return fail(TSDFS_E_INVALID, "mlp is NULL");
    if (m->arch != TSDFS_ARCH_TINY && m->arch != TSDFS_ARCH_ROOM) return fail(TSDFS_E_INVALID, "unknown arch %d", m->arch);
    if (m->precision != TSDFS_PREC_F32 && m->precision != TSDFS_PREC_BF16 && m->precision != TSDFS_PREC_F16 &&
        m->precision != TSDFS_PREC_BF16X2)
        return fail(TSDFS_E_INVALID, "unknown precision %d", m->precision);
    if (!m->sdf_w || !m->rgb_w) return fail(TSDFS_E_INVALID, "sdf_w and rgb_w must be non-NULL");
    if (!(m->scale > 0.0f) || !(m->beta > 0.0f) || !(m->inv_s > 0.0f) || !(m->alpha_eps >= 0.0f))
        return fail(TSDFS_E_INVALID, "scale, beta and inv_s must be > 0, alpha_eps >= 0");
    if (m->opacity != TSDFS_OPACITY_NEUS && m->opacity != TSDFS_OPACITY_VOLSDF)
        return fail(TSDFS_E_INVALID, "unknown opacity %d", m->opacity);
    if (m->precision != TSDFS_PREC_F32) {
        if (!m->packed) return fail(TSDFS_E_INVALID, "16-bit precisions need packed weights (tsdfs_pack_mlp)");
        if (!mlp_tc_available(m->arch)) return fail(TSDFS_E_UNSUPPORTED, "BF16 tensor-core path not available for arch %d", m->arch);
    }
    return TSDFS_OK;
}

static Opacity opacity_of(const tsdfs_mlp* m) { return Opacity{m->opacity, m->inv_s, m->alpha_eps}; }

static NetParams net_params(const tsdfs_mlp* m) {
    NetParams np;
    np.sdf_w = m->sdf_w;
    np.rgb_w = m->rgb_w;
    for (int a = 0; a < 3; ++a) np.center[a] = m->center[a];
    np.scale = m->scale;
    np.inv_scale = 1.0f / m->scale;
    np.beta = m->beta;
    return np;
}

// the network evaluation of every render path; `stash`: the serial tensor-core kernel's parking
// space in the caller's workspace (mlp_tc_stash_bytes(), 256-byte aligned)
static int run_full_mlp(const tsdfs_mlp* m, const SampleSource& src, SampleRec* rec, int64_t max_samples,
                        uint8_t* stash, cudaStream_t st) {
    if (m->precision != TSDFS_PREC_F32) {
        if (netkernel_of(m->precision) == TSDFS_NETKERNEL_PIPELINED) {
            ProfScope ps("mlp_pipe", st);
            return launch_mlp_pipe(m, src, rec, max_samples, st);
        }
        ProfScope ps("mlp_tc", st);
        return launch_mlp_full_tc(m, src, rec, max_samples, stash, st);
    }
    ProfScope ps("mlp_simt", st);
    const NetParams np = net_params(m);
    return m->arch == TSDFS_ARCH_TINY ? launch_mlp_full_simt<TSDFS_ARCH_TINY>(np, src, rec, max_samples, st)
                                      : launch_mlp_full_simt<TSDFS_ARCH_ROOM>(np, src, rec, max_samples, st);
}

}  // namespace tsdfs

using namespace tsdfs;

extern "C" const char* tsdfs_last_error(void) { return g_msg; }

extern "C" int tsdfs_set_test_limits(uint32_t spin_limit, int32_t march_step_cap, int32_t withhold_chunk) {
    if (march_step_cap < 0) return fail(TSDFS_E_INVALID, "tsdfs_set_test_limits: march_step_cap must be >= 0");
    if (withhold_chunk < -1) return fail(TSDFS_E_INVALID, "tsdfs_set_test_limits: withhold_chunk must be >= -1");
    g_test_spin.store(spin_limit);
    g_test_march.store(march_step_cap);
    g_test_withhold.store(withhold_chunk);
    return TSDFS_OK;
}

extern "C" int tsdfs_set_network_kernel(int32_t precision, int32_t kernel) {
    if (precision != TSDFS_PREC_BF16 && precision != TSDFS_PREC_F16 && precision != TSDFS_PREC_BF16X2)
        return fail(TSDFS_E_INVALID, "tsdfs_set_network_kernel: precision %d has no tensor-core kernel", precision);
    if (kernel != TSDFS_NETKERNEL_SERIAL && kernel != TSDFS_NETKERNEL_PIPELINED)
        return fail(TSDFS_E_INVALID, "tsdfs_set_network_kernel: unknown kernel %d", kernel);
    if (precision == TSDFS_PREC_BF16X2 && kernel != TSDFS_NETKERNEL_PIPELINED)
        return fail(TSDFS_E_INVALID, "tsdfs_set_network_kernel: BF16X2 runs on the pipelined kernel only");
    std::lock_guard<std::mutex> lk(g_netkernel_mu);
    g_netkernel[precision] = kernel;
    return TSDFS_OK;
}

extern "C" int tsdfs_network_kernel(int32_t precision) {
    if (precision != TSDFS_PREC_BF16 && precision != TSDFS_PREC_F16 && precision != TSDFS_PREC_BF16X2)
        return fail(TSDFS_E_INVALID, "tsdfs_network_kernel: precision %d has no tensor-core kernel", precision);
    return netkernel_of(precision);
}

extern "C" int tsdfs_profile(int32_t enable) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_clear();
    g_prof_on = enable != 0;
    return TSDFS_OK;
}

extern "C" int tsdfs_profile_read(const char* prefix, double* total_ms, int64_t* launches) {
    if (!total_ms || !launches) return fail(TSDFS_E_INVALID, "total_ms and launches must be non-NULL");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    double ms = 0.0;
    int64_t n = 0;
    const size_t plen = prefix ? strlen(prefix) : 0;
    for (size_t i = 0; i < g_prof_n; ++i) {
        if (plen && strncmp(g_prof[i].name, prefix, plen) != 0) continue;
        int rc = cuda_check(cudaEventSynchronize(g_prof[i].b), "tsdfs_profile_read synchronize");
        if (rc) return rc;
        float e = 0.0f;
        rc = cuda_check(cudaEventElapsedTime(&e, g_prof[i].a, g_prof[i].b), "tsdfs_profile_read elapsed");
        if (rc) return rc;
        ms += e;
        ++n;
    }
    *total_ms = ms;
    *launches = n;
    return TSDFS_OK;
}

extern "C" int tsdfs_sync_status(tsdfs_stream_t stream, uint32_t* bits_out) {
    int rc = cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "tsdfs_sync_status synchronize");
    if (rc) return rc;
    uint32_t bits = 0;
    rc = cuda_check(cudaMemcpyFromSymbol(&bits, g_status_word, sizeof bits), "tsdfs_sync_status read");
    if (rc) return rc;
    const uint32_t zero = 0;
    rc = cuda_check(cudaMemcpyToSymbol(g_status_word, &zero, sizeof zero), "tsdfs_sync_status clear");
    if (rc) return rc;
    if (bits_out) *bits_out = bits;
    if (bits) return fail(TSDFS_E_DEVICE, "device status bits 0x%x", bits);
    return TSDFS_OK;
}

extern "C" int64_t tsdfs_sdf_param_count(int32_t arch) {
    return arch == TSDFS_ARCH_TINY ? sdf_param_count<TSDFS_ARCH_TINY>()
                                   : (arch == TSDFS_ARCH_ROOM ? sdf_param_count<TSDFS_ARCH_ROOM>() : -1);
}
extern "C" int64_t tsdfs_rgb_param_count(int32_t arch) {
    return arch == TSDFS_ARCH_TINY ? rgb_param_count<TSDFS_ARCH_TINY>()
                                   : (arch == TSDFS_ARCH_ROOM ? rgb_param_count<TSDFS_ARCH_ROOM>() : -1);
}

// render workspace: the per-sample records, then the ray index of every sample, then the
// tensor-core network kernel's parking space
extern "C" size_t tsdfs_render_workspace_size(const tsdfs_mlp* mlp, int64_t n_rays, int64_t max_samples) {
    (void)mlp;
    (void)n_rays;
    if (max_samples < 0) return 0;
    return align256((size_t)max_samples * sizeof(SampleRec)) + align256((size_t)max_samples * sizeof(int32_t)) +
           align256(mlp_tc_stash_bytes()) + 256;
}

namespace tsdfs {
// ray index of every sample: thread r writes r into offsets[r] .. offsets[r+1] - 1
// (nothing at or beyond capacity: the network kernel flags that overflow itself)
__global__ void k_sample_ray(const int32_t* __restrict__ offsets, int64_t n_rays, int64_t capacity,
                             int32_t* __restrict__ sample_ray) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rays; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o0 = offsets[r], o1 = offsets[r + 1] < capacity ? offsets[r + 1] : capacity;
        for (int64_t i = o0; i < o1; ++i) sample_ray[i] = (int32_t)r;
    }
}
}  // namespace tsdfs

extern "C" int render_rays(const tsdfs_mlp* mlp, const float* ray_o, const float* ray_d, const float* t_n,
                           const float* t_f, const int32_t* offsets, const uint8_t* status, int64_t n_rays,
                           int64_t max_samples, float* rgb, float* depth, float* wsum, float* normal, float* eik,
                           void* ws, size_t ws_bytes, tsdfs_stream_t stream) {
    int rc = mlp_check(mlp);
    if (rc) return rc;
    if (n_rays < 0 || max_samples < 0) return fail(TSDFS_E_INVALID, "n_rays and max_samples must be >= 0");
    if (n_rays == 0) return TSDFS_OK;
    if (!ray_o || !ray_d || !t_n || !t_f || !offsets || !status || !rgb || !depth || !wsum)
        return fail(TSDFS_E_INVALID, "ray, bound and output pointers must be non-NULL (normal, eik may be NULL)");
    if (max_samples > (int64_t)INT32_MAX) return fail(TSDFS_E_INVALID, "max_samples must fit int32 offsets");
    if (!ws || ws_bytes < tsdfs_render_workspace_size(mlp, n_rays, max_samples))
        return fail(TSDFS_E_WORKSPACE, "render workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    SampleRec* rec = reinterpret_cast<SampleRec*>((reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255));
    int32_t* sample_ray = reinterpret_cast<int32_t*>(reinterpret_cast<uintptr_t>(rec) +
                                                     align256((size_t)max_samples * sizeof(SampleRec)));
    uint8_t* stash = reinterpret_cast<uint8_t*>(reinterpret_cast<uintptr_t>(sample_ray) +
                                                align256((size_t)max_samples * sizeof(int32_t)));
    SampleSource src{};
    src.mode = kUniform;
    src.ray_o = ray_o;
    src.ray_d = ray_d;
    src.offsets = offsets;
    src.t_n = t_n;
    src.t_f = t_f;
    src.n_rays = n_rays;
    src.total_dev = offsets + n_rays;
    src.capacity = max_samples;
    if (max_samples > 0) {
        if (mlp->precision != TSDFS_PREC_F32) {
            ProfScope ps("sample_ray", st);
            k_sample_ray<<<grid_1d(n_rays, 256), 256, 0, st>>>(offsets, n_rays, max_samples, sample_ray);
            rc = cuda_check(cudaGetLastError(), "sample_ray launch");
            if (rc) return rc;
            src.sample_ray = sample_ray;
        }
        rc = run_full_mlp(mlp, src, rec, max_samples, stash, st);
        if (rc) return rc;
    }
    ProfScope ps("composite", st);
    return launch_composite(rec, offsets, 0, status, n_rays, offsets + n_rays, max_samples, opacity_of(mlp),
                            rgb, depth, wsum, normal, eik, st);
}

extern "C" int tsdfs_autotune_network(const tsdfs_mlp* mlp, const float* ray_o, const float* ray_d, const float* t_n,
                                      const float* t_f, const int32_t* offsets, const uint8_t* status, int64_t n_rays,
                                      int64_t max_samples, float* rgb, float* depth, float* wsum, float* normal,
                                      void* ws, size_t ws_bytes, int32_t reps, float* ms_out,
                                      tsdfs_stream_t stream) {
    int rc = mlp_check(mlp);
    if (rc) return rc;
    if (mlp->precision == TSDFS_PREC_F32) return fail(TSDFS_E_INVALID, "tsdfs_autotune_network: FP32 has one kernel");
    if (reps < 1) return fail(TSDFS_E_INVALID, "tsdfs_autotune_network: reps must be >= 1");
    const int cands[2] = {TSDFS_NETKERNEL_SERIAL, TSDFS_NETKERNEL_PIPELINED};
    float best_ms = 0.0f;
    int best = TSDFS_NETKERNEL_PIPELINED;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rc = cuda_check(cudaEventCreate(&e0), "autotune_network event");
    if (!rc) rc = cuda_check(cudaEventCreate(&e1), "autotune_network event");
    const int old = netkernel_of(mlp->precision);
    for (int c = 0; c < 2 && !rc; ++c) {
        float ms = -1.0f;
        if (cands[c] == TSDFS_NETKERNEL_SERIAL && mlp->precision == TSDFS_PREC_BF16X2) {
            if (ms_out) ms_out[c] = ms;
            continue;
        }
        {
            std::lock_guard<std::mutex> lk(g_netkernel_mu);
            g_netkernel[mlp->precision] = cands[c];
        }
        rc = render_rays(mlp, ray_o, ray_d, t_n, t_f, offsets, status, n_rays, max_samples, rgb, depth, wsum, normal,
                         nullptr, ws, ws_bytes, stream);
        if (!rc) rc = cuda_check(cudaEventRecord(e0, st), "autotune_network record");
        for (int r = 0; r < reps && !rc; ++r)
            rc = render_rays(mlp, ray_o, ray_d, t_n, t_f, offsets, status, n_rays, max_samples, rgb, depth, wsum,
                             normal, nullptr, ws, ws_bytes, stream);
        if (!rc) rc = cuda_check(cudaEventRecord(e1, st), "autotune_network record");
        if (!rc) rc = cuda_check(cudaEventSynchronize(e1), "autotune_network sync");
        if (!rc) rc = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "autotune_network elapsed");
        if (rc) break;
        ms /= (float)reps;
        if (ms_out) ms_out[c] = ms;
        if (best_ms == 0.0f || ms < best_ms) {
            best_ms = ms;
            best = cands[c];
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(g_netkernel_mu);
    g_netkernel[mlp->precision] = rc ? old : best;
    return rc ? rc : best;
}

// ---- hierarchical comparator ------------------------------------------------
struct HierWs {
    float *t0, *te, *tc, *dc, *fc, *tf, *df;
    uint8_t* status;
    SampleRec* rec;
    uint8_t* stash;
    size_t bytes;
};

static HierWs hier_layout(void* base, int64_t n, int n_c = 64, int n_f = 32) {
    HierWs w{};
    uintptr_t p = (reinterpret_cast<uintptr_t>(base) + 255) & ~uintptr_t(255);
    auto take = [&](size_t bytes) {
        uintptr_t q = p;
        p = (p + bytes + 255) & ~uintptr_t(255);
        return q;
    };
    const size_t n_h = (size_t)(n_c + n_f);
    w.rec = reinterpret_cast<SampleRec*>(take((size_t)n * n_h * sizeof(SampleRec)));
    w.stash = reinterpret_cast<uint8_t*>(take(mlp_tc_stash_bytes()));
    w.t0 = reinterpret_cast<float*>(take((size_t)n * 4));
    w.te = reinterpret_cast<float*>(take((size_t)n * 4));
    w.tc = reinterpret_cast<float*>(take((size_t)n * n_c * 4));
    w.dc = reinterpret_cast<float*>(take((size_t)n * n_c * 4));
    w.fc = reinterpret_cast<float*>(take((size_t)n * n_c * 4));
    w.tf = reinterpret_cast<float*>(take((size_t)n * n_h * 4));
    w.df = reinterpret_cast<float*>(take((size_t)n * n_h * 4));
    w.status = reinterpret_cast<uint8_t*>(take((size_t)n));
    w.bytes = p - reinterpret_cast<uintptr_t>(base) + 256;
    return w;
}

extern "C" size_t tsdfs_hier_workspace_size(const tsdfs_mlp* mlp, int64_t n_rays) {
    (void)mlp;
    if (n_rays < 0) return 0;
    return hier_layout(nullptr, n_rays).bytes + 256;
}

extern "C" int render_rays_hier(const tsdfs_mlp* mlp, const tsdfs_grid* grid, const float* ray_o, const float* ray_d,
                                int64_t n_rays, int n_coarse, int n_fine, float t_near, float t_far, float* rgb,
                                float* depth, float* wsum, float* normal, void* ws, size_t ws_bytes,
                                tsdfs_stream_t stream) {
    int rc = mlp_check(mlp);
    if (rc) return rc;
    if (!grid) return fail(TSDFS_E_INVALID, "grid is NULL");
    if (grid->nx <= 0 || grid->ny <= 0 || grid->nz <= 0 || !(grid->voxel_size > 0.0f))
        return fail(TSDFS_E_INVALID, "grid geometry invalid");
    if (n_coarse < 2 || n_coarse > 64 || n_fine < 1 || n_fine > 32)
        return fail(TSDFS_E_INVALID, "sample counts must be coarse in [2, 64], fine in [1, 32]");
    if (n_rays < 0) return fail(TSDFS_E_INVALID, "n_rays must be >= 0");
    if (n_rays == 0) return TSDFS_OK;
    const int n_h = n_coarse + n_fine;
    if (n_rays * 96 > (int64_t)INT32_MAX) return fail(TSDFS_E_INVALID, "too many rays");
    if (!ray_o || !ray_d || !rgb || !depth || !wsum) return fail(TSDFS_E_INVALID, "ray and output pointers must be non-NULL");
    if (!(t_near < t_far)) return fail(TSDFS_E_INVALID, "t_near must be < t_far");
    if (!ws || ws_bytes < tsdfs_hier_workspace_size(mlp, n_rays)) return fail(TSDFS_E_WORKSPACE, "hier workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    HierWs w = hier_layout(ws, n_rays, n_coarse, n_fine);
    {
        ProfScope ps("hier_setup", st);
        rc = launch_hier_setup(grid, ray_o, ray_d, n_rays, t_near, t_far, w.t0, w.te, w.status, w.tc, w.dc, n_coarse, st);
    }
    if (rc) return rc;
    const NetParams np = net_params(mlp);
    SampleSource cs{};
    cs.mode = kExplicit;
    cs.ray_o = ray_o;
    cs.ray_d = ray_d;
    cs.t = w.tc;
    cs.delta = w.dc;
    cs.per_ray = n_coarse;
    cs.total_host = n_rays * n_coarse;
    cs.capacity = n_rays * n_coarse;
    if (mlp->precision != TSDFS_PREC_F32) {
        ProfScope ps("mlp_value_tc", st);
        rc = launch_mlp_value_tc(mlp, cs, w.fc, st);
    } else {
        ProfScope ps("mlp_value_simt", st);
        rc = mlp->arch == TSDFS_ARCH_TINY ? launch_mlp_value_simt<TSDFS_ARCH_TINY>(np, cs, w.fc, st)
                                          : launch_mlp_value_simt<TSDFS_ARCH_ROOM>(np, cs, w.fc, st);
    }
    if (rc) return rc;
    {
        ProfScope ps("hier_fine", st);
        rc = launch_hier_fine(w.fc, w.tc, w.t0, w.te, n_rays, opacity_of(mlp), w.tf, w.df, n_coarse, n_fine,
                              st);
    }
    if (rc) return rc;
    SampleSource fs = cs;
    fs.t = w.tf;
    fs.delta = w.df;
    fs.per_ray = n_h;
    fs.total_host = n_rays * n_h;
    fs.capacity = n_rays * n_h;
    rc = run_full_mlp(mlp, fs, w.rec, n_rays * n_h, w.stash, st);
    if (rc) return rc;
    ProfScope ps("composite", st);
    return launch_composite(w.rec, nullptr, n_h, w.status, n_rays, nullptr, n_rays * n_h, opacity_of(mlp),
                            rgb, depth, wsum, normal, nullptr, st);
}

extern "C" int render_rays_hier96(const tsdfs_mlp* mlp, const tsdfs_grid* grid, const float* ray_o,
                                  const float* ray_d, int64_t n_rays, float t_near, float t_far, float* rgb,
                                  float* depth, float* wsum, float* normal, void* ws, size_t ws_bytes,
                                  tsdfs_stream_t stream) {
    return render_rays_hier(mlp, grid, ray_o, ray_d, n_rays, 64, 32, t_near, t_far, rgb, depth, wsum, normal, ws,
                            ws_bytes, stream);
}

// ---- coarse + fine inside the TSDF bound ----------------------------------------
struct BoundedHierWs {
    int32_t *ray_c, *n2, *off2, *sums, *ray2;
    float *fc, *t2, *d2;
    SampleRec* rec;
    uint8_t* stash;
    size_t bytes;
};

static BoundedHierWs bounded_hier_layout(void* base, int64_t n, int64_t max_coarse, int64_t cap2) {
    BoundedHierWs w{};
    uintptr_t p = (reinterpret_cast<uintptr_t>(base) + 255) & ~uintptr_t(255);
    auto take = [&](size_t bytes) {
        uintptr_t q = p;
        p = (p + bytes + 255) & ~uintptr_t(255);
        return q;
    };
    w.rec = reinterpret_cast<SampleRec*>(take((size_t)cap2 * sizeof(SampleRec)));
    w.stash = reinterpret_cast<uint8_t*>(take(mlp_tc_stash_bytes()));
    w.ray_c = reinterpret_cast<int32_t*>(take((size_t)max_coarse * 4));
    w.fc = reinterpret_cast<float*>(take((size_t)max_coarse * 4));
    w.n2 = reinterpret_cast<int32_t*>(take((size_t)n * 4));
    w.off2 = reinterpret_cast<int32_t*>(take((size_t)(n + 1) * 4));
    w.sums = reinterpret_cast<int32_t*>(take((size_t)(scan_chunks(n) + 1) * 4));
    w.t2 = reinterpret_cast<float*>(take((size_t)cap2 * 4));
    w.d2 = reinterpret_cast<float*>(take((size_t)cap2 * 4));
    w.ray2 = reinterpret_cast<int32_t*>(take((size_t)cap2 * 4));
    w.bytes = p - reinterpret_cast<uintptr_t>(base) + 256;
    return w;
}

extern "C" size_t tsdfs_hier_bounded_workspace_size(const tsdfs_mlp* mlp, int64_t n_rays, int32_t n_fine,
                                                    int64_t max_coarse) {
    (void)mlp;
    if (n_rays < 0 || max_coarse < 0 || n_fine < 0) return 0;
    return bounded_hier_layout(nullptr, n_rays, max_coarse, max_coarse + n_rays * n_fine).bytes + 256;
}

extern "C" int render_rays_hier_bounded(const tsdfs_mlp* mlp, const float* ray_o, const float* ray_d,
                                        const float* t_n, const float* t_f, const int32_t* offsets,
                                        const uint8_t* status, int64_t n_rays, int32_t n_fine, int64_t max_coarse,
                                        float* rgb, float* depth, float* wsum, float* normal, void* ws,
                                        size_t ws_bytes, tsdfs_stream_t stream) {
    int rc = mlp_check(mlp);
    if (rc) return rc;
    if (n_rays < 0 || max_coarse < 0) return fail(TSDFS_E_INVALID, "n_rays and max_coarse must be >= 0");
    if (n_fine < 0 || n_fine > 32) return fail(TSDFS_E_INVALID, "fine sample count must be in [0, 32]");
    if (n_rays == 0) return TSDFS_OK;
    const int64_t cap2 = max_coarse + n_rays * (int64_t)n_fine;
    if (cap2 > (int64_t)INT32_MAX) return fail(TSDFS_E_INVALID, "max_coarse + n_rays * n_fine must fit int32 offsets");
    if (!ray_o || !ray_d || !t_n || !t_f || !offsets || !status || !rgb || !depth || !wsum)
        return fail(TSDFS_E_INVALID, "ray, bound and output pointers must be non-NULL (normal may be NULL)");
    if (!ws || ws_bytes < tsdfs_hier_bounded_workspace_size(mlp, n_rays, n_fine, max_coarse))
        return fail(TSDFS_E_WORKSPACE, "bounded hierarchical workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    BoundedHierWs w = bounded_hier_layout(ws, n_rays, max_coarse, cap2);
    // coarse pass: SDF values at the midpoints of the bounds' ragged counts
    SampleSource cs{};
    cs.mode = kUniform;
    cs.ray_o = ray_o;
    cs.ray_d = ray_d;
    cs.offsets = offsets;
    cs.t_n = t_n;
    cs.t_f = t_f;
    cs.n_rays = n_rays;
    cs.total_dev = offsets + n_rays;
    cs.capacity = max_coarse;
    {
        {
            ProfScope ps("sample_ray", st);
            k_sample_ray<<<grid_1d(n_rays, 256), 256, 0, st>>>(offsets, n_rays, max_coarse, w.ray_c);
            rc = cuda_check(cudaGetLastError(), "sample_ray launch");
            if (rc) return rc;
        }
        cs.sample_ray = w.ray_c;  // the value kernels flag a coarse total above max_coarse
        if (mlp->precision != TSDFS_PREC_F32) {
            ProfScope ps("mlp_value_tc", st);
            rc = launch_mlp_value_tc(mlp, cs, w.fc, st);
        } else {
            ProfScope ps("mlp_value_simt", st);
            const NetParams np = net_params(mlp);
            rc = mlp->arch == TSDFS_ARCH_TINY ? launch_mlp_value_simt<TSDFS_ARCH_TINY>(np, cs, w.fc, st)
                                              : launch_mlp_value_simt<TSDFS_ARCH_ROOM>(np, cs, w.fc, st);
        }
        if (rc) return rc;
    }
    // merged counts, their offsets, then the fine samples and the merged list
    {
        ProfScope ps("bounded_fine", st);
        rc = launch_bounded_counts(offsets, n_rays, n_fine, max_coarse, w.n2, st);
        if (rc) return rc;
        rc = exclusive_scan(w.n2, n_rays, w.off2, w.sums, st);
        if (rc) return rc;
        rc = launch_bounded_fine(w.fc, offsets, t_n, t_f, w.off2, n_rays, n_fine, opacity_of(mlp),
                                 max_coarse, cap2, w.t2, w.d2, w.ray2, st);
        if (rc) return rc;
    }
    SampleSource fs{};
    fs.mode = kExplicit;
    fs.ray_o = ray_o;
    fs.ray_d = ray_d;
    fs.t = w.t2;
    fs.delta = w.d2;
    fs.sample_ray = w.ray2;
    fs.per_ray = 1;
    fs.n_rays = n_rays;
    fs.total_dev = w.off2 + n_rays;
    fs.capacity = cap2;
    if (cap2 > 0) {
        rc = run_full_mlp(mlp, fs, w.rec, cap2, w.stash, st);
        if (rc) return rc;
    }
    ProfScope ps("composite", st);
    return launch_composite(w.rec, w.off2, 0, status, n_rays, w.off2 + n_rays, cap2, opacity_of(mlp), rgb,
                            depth, wsum, normal, nullptr, st);
}
