// K3: TSDF sample bounds of Alg. 1 + the adaptive count of Sec. 3.4.
// K4: exclusive scan of the counts into ragged offsets.
//
// One thread per ray; the voxel walk recomputes every crossing parameter from
// its integer boundary, so the walk is exact to the voxel no matter how long.
// fp32, round-to-nearest, no contraction (intrinsics + --fmad=false), in the
// operation order of the oracle's fp32-exact mode, so t_n, t_f, counts and
// status are identical bit for bit.
#include <mutex>

#include "common.cuh"
#include "march.cuh"

namespace tsdfs {
int grid_check(const tsdfs_grid* g);

namespace {

constexpr int kBoundsBlock = 128;      // default threads per block of the march
constexpr int kBoundsMaxBlock = 256;   // largest block the autotuner may pick
constexpr int kScanBlock = 1024;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanBlock * kScanItems;

struct BoundsDev {
    float d_s, t_near, t_far, step;
    int nb_radius, m_confirm, n_max, n_fallback;
    int max_steps;   // voxel steps a walk may take (0: nx + ny + nz + 8, more than any walk needs)
};

__device__ __forceinline__ float trilinear(const GridDev& g, const float p[3]) {
    int i0[3];
    float fr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float gg = __fsub_rn(__fdiv_rn(__fsub_rn(p[a], g.org[a]), g.vs), 0.5f);
        float fl = floorf(gg);
        fr[a] = __fsub_rn(gg, fl);
        if (!(fl >= -1.0f)) { fl = -1.0f; fr[a] = 1.0f; }
        if (fl > (float)g.n[a]) { fl = (float)g.n[a]; fr[a] = 0.0f; }
        i0[a] = (int)fl;
    }
    float c[2][2][2];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const int ii = min(max(i0[0] + dx, 0), g.n[0] - 1);
                const int jj = min(max(i0[1] + dy, 0), g.n[1] - 1);
                const int kk = min(max(i0[2] + dz, 0), g.n[2] - 1);
                c[dz][dy][dx] = gval(g, ii, jj, kk);
            }
    const float x00 = __fadd_rn(c[0][0][0], __fmul_rn(fr[0], __fsub_rn(c[0][0][1], c[0][0][0])));
    const float x01 = __fadd_rn(c[0][1][0], __fmul_rn(fr[0], __fsub_rn(c[0][1][1], c[0][1][0])));
    const float x10 = __fadd_rn(c[1][0][0], __fmul_rn(fr[0], __fsub_rn(c[1][0][1], c[1][0][0])));
    const float x11 = __fadd_rn(c[1][1][0], __fmul_rn(fr[0], __fsub_rn(c[1][1][1], c[1][1][0])));
    const float y0 = __fadd_rn(x00, __fmul_rn(fr[1], __fsub_rn(x01, x00)));
    const float y1 = __fadd_rn(x10, __fmul_rn(fr[1], __fsub_rn(x11, x10)));
    return __fadd_rn(y0, __fmul_rn(fr[2], __fsub_rn(y1, y0)));
}

__device__ __forceinline__ bool all_negative(const GridDev& g, const int X[3], int r) {
    for (int dz = -r; dz <= r; ++dz)
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx)
                if (!(gval(g, X[0] + dx, X[1] + dy, X[2] + dz) < 0.0f)) return false;
    return true;
}

__device__ __forceinline__ bool inside_bit(const uint32_t* __restrict__ mask, const GridDev& g, const int X[3]) {
    const int64_t idx = ((int64_t)X[2] * g.n[1] + X[1]) * g.n[0] + X[0];
    return (__ldg(mask + (idx >> 5)) >> (idx & 31)) & 1u;
}

__global__ void __launch_bounds__(kBoundsMaxBlock) k_ray_bounds(GridDev g, const uint32_t* __restrict__ mask,
                                                             const float* __restrict__ ray_o,
                                                             const float* __restrict__ ray_d, int64_t n_rays,
                                                             BoundsDev p, float* __restrict__ t_n_out,
                                                             float* __restrict__ t_f_out, int32_t* __restrict__ n_out,
                                                             float* __restrict__ t_zero_out,
                                                             uint8_t* __restrict__ status_out, uint32_t* dev_status) {
    const float kInf = __int_as_float(0x7f800000);
    const float kNaN = __int_as_float(0x7fffffff);
    const float ds_norm = __fdiv_rn(p.d_s, g.trunc);
    const int max_steps = p.max_steps > 0 ? p.max_steps : g.n[0] + g.n[1] + g.n[2] + 8;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rays; r += (int64_t)gridDim.x * blockDim.x) {
        float o[3], d[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = __ldg(ray_o + 3 * r + a);
            d[a] = __ldg(ray_d + 3 * r + a);
        }
        // ---- clip to the grid box ("RenderingCube") ----
        float t0, t_end;
        if (!clip_box(g, o, d, p.t_near, p.t_far, t0, t_end)) {
            t_n_out[r] = 0.0f; t_f_out[r] = 0.0f; n_out[r] = 0; status_out[r] = TSDFS_MISS;
            if (t_zero_out) t_zero_out[r] = kNaN;
            continue;
        }
        // ---- voxel walk init ----
        Dda s;
        dda_init(s, g, o, d, t0);
        // ---- near phase: first voxel with V(centre) <= D_s ----
        // The walk does not depend on the values: the next kAhead voxels are stepped and
        // their values requested before the current one is tested, so the loads are in
        // flight together; the voxels, their order and every test are unchanged.
        constexpr int kAhead = 4;
        Dda wq[kAhead];
        float qv[kAhead];
        bool qok[kAhead];   // the loop condition of that step: still in the grid, t < t_end
        bool live = true;   // the walk has not left the grid
        wq[0] = s;
        qok[0] = s.t < t_end;
        qv[0] = gval(g, s.X[0], s.X[1], s.X[2]);
#pragma unroll
        for (int i = 1; i < kAhead; ++i) {
            wq[i] = wq[i - 1];
            live = live && dda_next(wq[i], g, o);
            qok[i] = live && wq[i].t < t_end;
            qv[i] = live ? gval(g, wq[i].X[0], wq[i].X[1], wq[i].X[2]) : 0.0f;
        }
        bool found = false, in_grid = true;
        float t_before = t0;
        int steps = 0;
        while (qok[0]) {
            if (++steps > max_steps) { set_status(dev_status, TSDFS_DEV_MARCH_CAP); in_grid = false; break; }
            if (qv[0] <= ds_norm) { found = true; break; }
            t_before = wq[0].t;
            Dda nx = wq[kAhead - 1];
#pragma unroll
            for (int i = 0; i + 1 < kAhead; ++i) {
                wq[i] = wq[i + 1];
                qv[i] = qv[i + 1];
                qok[i] = qok[i + 1];
            }
            live = live && dda_next(nx, g, o);
            wq[kAhead - 1] = nx;
            qok[kAhead - 1] = live && nx.t < t_end;
            qv[kAhead - 1] = live ? gval(g, nx.X[0], nx.X[1], nx.X[2]) : 0.0f;
        }
        s = wq[0];
        if (!found) {
            t_n_out[r] = t0; t_f_out[r] = t_end; n_out[r] = p.n_fallback; status_out[r] = TSDFS_FALLBACK;
            if (t_zero_out) t_zero_out[r] = kNaN;
            continue;
        }
        const float tn = s.t;
        float tf = t_end;
        // ---- zero-crossing search, starting at the entry of the voxel before ----
        float tz = kNaN, t_prev = t_before, v_prev;
        {
            float pp[3];
            point_at(o, d, t_before, pp);
            v_prev = trilinear(g, pp);
            point_at(o, d, tn, pp);
            const float vn = trilinear(g, pp);
            if (tn > t_before && v_prev > 0.0f && vn <= 0.0f)
                tz = __fadd_rn(t_prev, __fmul_rn(__fsub_rn(tn, t_prev), __fdiv_rn(v_prev, __fsub_rn(v_prev, vn))));
            v_prev = vn;
            t_prev = tn;
        }
        // ---- far phase: consecutive voxels whose neighbourhood is all negative ----
        int m = 0;
        while (in_grid && s.t < t_end) {
            if (++steps > max_steps) { set_status(dev_status, TSDFS_DEV_MARCH_CAP); break; }
            const bool inside = mask ? inside_bit(mask, g, s.X) : all_negative(g, s.X, p.nb_radius);
            m = inside ? m + 1 : 0;
            in_grid = dda_next(s, g, o);
            const float tc = s.t < t_end ? s.t : t_end;
            if (tz != tz) {
                float pp[3];
                point_at(o, d, tc, pp);
                const float vc = trilinear(g, pp);
                if (v_prev > 0.0f && vc <= 0.0f)
                    tz = __fadd_rn(t_prev, __fmul_rn(__fsub_rn(tc, t_prev), __fdiv_rn(v_prev, __fsub_rn(v_prev, vc))));
                v_prev = vc;
                t_prev = tc;
            }
            if (m == p.m_confirm) { tf = tc; break; }
        }
        // ---- adaptive count (Sec. 3.4) ----
        const float q = __fdiv_rn(__fsub_rn(tf, tn), p.step);
        int cnt;
        if (!(q > 1.0f)) cnt = 1;
        else if (q >= (float)p.n_max) cnt = p.n_max;
        else cnt = (int)ceilf(q);
        if (cnt > p.n_max) cnt = p.n_max;
        t_n_out[r] = tn; t_f_out[r] = tf; n_out[r] = cnt; status_out[r] = TSDFS_BOUNDED;
        if (t_zero_out) t_zero_out[r] = tz;
    }
}

// ---- recovery (Sec. 4.5): BOUNDED rays whose weight sum stayed below tau are
// rendered again over the whole [t0, t_end] with n_fallback samples ----
__global__ void __launch_bounds__(kBoundsMaxBlock) k_recovery_bounds(GridDev g, const float* __restrict__ ray_o,
                                                                  const float* __restrict__ ray_d, int64_t n_rays,
                                                                  BoundsDev p, float tau,
                                                                  const float* __restrict__ wsum,
                                                                  const uint8_t* __restrict__ status,
                                                                  float* __restrict__ t_n2, float* __restrict__ t_f2,
                                                                  int32_t* __restrict__ n2, uint8_t* __restrict__ status2) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rays; r += (int64_t)gridDim.x * blockDim.x) {
        float o[3], d[3], t0 = 0.0f, t_end = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = __ldg(ray_o + 3 * r + a);
            d[a] = __ldg(ray_d + 3 * r + a);
        }
        const bool again = status[r] == TSDFS_BOUNDED && wsum[r] < tau && clip_box(g, o, d, p.t_near, p.t_far, t0, t_end);
        t_n2[r] = again ? t0 : 0.0f;
        t_f2[r] = again ? t_end : 0.0f;
        n2[r] = again ? p.n_fallback : 0;
        status2[r] = again ? (uint8_t)TSDFS_FALLBACK : (uint8_t)TSDFS_MISS;
    }
}

// ---- K4: three-phase exclusive scan (chunk sums, scan of sums, chunk scan) ----
__device__ __forceinline__ int block_exclusive_scan(int v, int* sh, int& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;  // inclusive warp prefix
    }
    __syncthreads();
    total = sh[(blockDim.x >> 5) - 1];
    const int excl = x - v + (warp > 0 ? sh[warp - 1] : 0);
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(kScanBlock) k_chunk_sums(const int32_t* __restrict__ cnt, int64_t n,
                                                           int32_t* __restrict__ sums) {
    __shared__ int sh[32];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    int v = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) v += cnt[base + i];
    int total;
    block_exclusive_scan(v, sh, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_sums(int32_t* __restrict__ sums, int64_t n_chunks,
                                                          int32_t* __restrict__ offsets_last, int64_t n_rays) {
    __shared__ int sh[32];
    const int per = (int)((n_chunks + kScanBlock - 1) / kScanBlock);
    const int64_t base = (int64_t)threadIdx.x * per;
    int v = 0;
    for (int i = 0; i < per; ++i)
        if (base + i < n_chunks) v += sums[base + i];
    int total;
    int run = block_exclusive_scan(v, sh, total);
    for (int i = 0; i < per; ++i)
        if (base + i < n_chunks) {
            int c = sums[base + i];
            sums[base + i] = run;
            run += c;
        }
    if (threadIdx.x == 0) offsets_last[n_rays] = total;
}

__global__ void __launch_bounds__(kScanBlock) k_chunk_scan(const int32_t* __restrict__ cnt, int64_t n,
                                                           const int32_t* __restrict__ sums,
                                                           int32_t* __restrict__ offsets) {
    __shared__ int sh[32];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? cnt[base + i] : 0;
        s += v[i];
    }
    int total;
    int run = block_exclusive_scan(s, sh, total) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) {
            offsets[base + i] = run;
            run += v[i];
        }
}

}  // namespace

int64_t scan_chunks(int64_t n) { return (n + kScanChunk - 1) / kScanChunk; }

// ---- launch shape of the march (threads per block, resident blocks per SM of the
// grid-stride grid): the default, or what tsdfs_autotune_bounds measured, per device
namespace {
struct MarchShape {
    int block = kBoundsBlock;
    int blocks_per_sm = 64;
};
std::mutex g_shape_mu;
MarchShape g_shape[64];

MarchShape march_shape() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MarchShape{};
    std::lock_guard<std::mutex> lk(g_shape_mu);
    return g_shape[dev];
}

unsigned march_grid(int64_t n_rays, const MarchShape& sh) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return grid_1d(n_rays, sh.block, sms * sh.blocks_per_sm);
}
}  // namespace

// exclusive scan of n counts into offsets[0..n]; `sums` needs scan_chunks(n) ints
int exclusive_scan(const int32_t* cnt, int64_t n, int32_t* offsets, int32_t* sums, cudaStream_t st) {
    const int64_t chunks = scan_chunks(n);
    if (n == 0) return cuda_check(cudaMemsetAsync(offsets, 0, sizeof(int32_t), st), "scan memset");
    if (chunks > (int64_t)kScanBlock * 64) return fail(TSDFS_E_INVALID, "too many rays for the scan (%lld)", (long long)n);
    ProfScope ps("scan", st);
    k_chunk_sums<<<(unsigned)chunks, kScanBlock, 0, st>>>(cnt, n, sums);
    k_scan_sums<<<1, kScanBlock, 0, st>>>(sums, chunks, offsets, n);
    k_chunk_scan<<<(unsigned)chunks, kScanBlock, 0, st>>>(cnt, n, sums, offsets);
    return cuda_check(cudaGetLastError(), "scan launch");
}

}  // namespace tsdfs

using namespace tsdfs;

extern "C" size_t tsdfs_bounds_workspace_size(int64_t n_rays) {
    if (n_rays < 0) return 0;
    return (size_t)(scan_chunks(n_rays) + 1) * sizeof(int32_t) + 256;
}

extern "C" int tsdf_ray_bounds(const tsdfs_grid* g, const uint32_t* mask, const float* ray_o, const float* ray_d,
                               int64_t n_rays, const tsdfs_bounds_params* p, float* t_n, float* t_f,
                               int32_t* n_samples, int32_t* offsets, float* t_zero, uint8_t* status, void* ws,
                               size_t ws_bytes, tsdfs_stream_t stream) {
    int rc = grid_check(g);
    if (rc) return rc;
    if (!p) return fail(TSDFS_E_INVALID, "params is NULL");
    if (n_rays < 0) return fail(TSDFS_E_INVALID, "n_rays must be >= 0");
    if (n_rays > (int64_t)INT32_MAX) return fail(TSDFS_E_INVALID, "n_rays must fit in int32 offsets");
    if (!(p->step > 0.0f) || !(p->d_s == p->d_s)) return fail(TSDFS_E_INVALID, "step must be > 0 and d_s finite");
    if (p->nb_radius < 0 || p->nb_radius > 4) return fail(TSDFS_E_INVALID, "nb_radius must be in [0, 4]");
    if (p->m_confirm < 1) return fail(TSDFS_E_INVALID, "m_confirm must be >= 1");
    if (p->n_max < 1 || p->n_fallback < 0 || p->n_max > 4096 || p->n_fallback > 4096)
        return fail(TSDFS_E_INVALID, "n_max must be in [1, 4096] and n_fallback in [0, 4096]");
    if ((int64_t)(p->n_max > p->n_fallback ? p->n_max : p->n_fallback) * n_rays > (int64_t)INT32_MAX)
        return fail(TSDFS_E_INVALID, "sample total could overflow int32 offsets");
    if (!(p->t_near < p->t_far)) return fail(TSDFS_E_INVALID, "t_near must be < t_far");
    if (n_rays > 0 && (!ray_o || !ray_d || !t_n || !t_f || !n_samples || !status))
        return fail(TSDFS_E_INVALID, "ray and output pointers must be non-NULL");
    if (!offsets) return fail(TSDFS_E_INVALID, "offsets is NULL");
    if (ws_bytes < tsdfs_bounds_workspace_size(n_rays) || !ws) return fail(TSDFS_E_WORKSPACE, "bounds workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    if (n_rays > 0) {
        GridDev gd{g->tsdf, g->dtype == TSDFS_F16, {g->nx, g->ny, g->nz}, {g->origin[0], g->origin[1], g->origin[2]},
                   g->voxel_size, g->trunc};
        BoundsDev bd{p->d_s, p->t_near, p->t_far, p->step, p->nb_radius, p->m_confirm, p->n_max, p->n_fallback,
                     test_march_cap()};
        const MarchShape sh = march_shape();
        ProfScope ps("ray_bounds", st);
        k_ray_bounds<<<march_grid(n_rays, sh), sh.block, 0, st>>>(gd, mask, ray_o, ray_d, n_rays, bd, t_n, t_f,
                                                                  n_samples, t_zero, status, device_status_word());
        rc = cuda_check(cudaGetLastError(), "tsdf_ray_bounds launch");
        if (rc) return rc;
    }
    int32_t* sums = reinterpret_cast<int32_t*>((reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255));
    return exclusive_scan(n_samples, n_rays, offsets, sums, st);
}

extern "C" int tsdf_recovery_bounds(const tsdfs_grid* g, const float* ray_o, const float* ray_d, int64_t n_rays,
                                    const tsdfs_bounds_params* p, float tau, const float* wsum, const uint8_t* status,
                                    float* t_n2, float* t_f2, int32_t* n2, int32_t* offsets2, uint8_t* status2,
                                    void* ws, size_t ws_bytes, tsdfs_stream_t stream) {
    int rc = grid_check(g);
    if (rc) return rc;
    if (!p) return fail(TSDFS_E_INVALID, "params is NULL");
    if (n_rays < 0 || n_rays > (int64_t)INT32_MAX) return fail(TSDFS_E_INVALID, "n_rays must be in [0, 2^31)");
    if (!(p->t_near < p->t_far)) return fail(TSDFS_E_INVALID, "t_near must be < t_far");
    if (p->n_fallback < 0 || p->n_fallback > 4096) return fail(TSDFS_E_INVALID, "n_fallback must be in [0, 4096]");
    if ((int64_t)p->n_fallback * n_rays > (int64_t)INT32_MAX)
        return fail(TSDFS_E_INVALID, "sample total could overflow int32 offsets");
    if (!(tau == tau)) return fail(TSDFS_E_INVALID, "tau must not be NaN");
    if (n_rays > 0 && (!ray_o || !ray_d || !wsum || !status || !t_n2 || !t_f2 || !n2 || !status2))
        return fail(TSDFS_E_INVALID, "ray, input and output pointers must be non-NULL");
    if (!offsets2) return fail(TSDFS_E_INVALID, "offsets2 is NULL");
    if (ws_bytes < tsdfs_bounds_workspace_size(n_rays) || !ws) return fail(TSDFS_E_WORKSPACE, "recovery workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    if (n_rays > 0) {
        GridDev gd{g->tsdf, g->dtype == TSDFS_F16, {g->nx, g->ny, g->nz}, {g->origin[0], g->origin[1], g->origin[2]},
                   g->voxel_size, g->trunc};
        BoundsDev bd{p->d_s, p->t_near, p->t_far, p->step, p->nb_radius, p->m_confirm, p->n_max, p->n_fallback,
                     test_march_cap()};
        const MarchShape sh = march_shape();
        ProfScope ps("recovery_bounds", st);
        k_recovery_bounds<<<march_grid(n_rays, sh), sh.block, 0, st>>>(
            gd, ray_o, ray_d, n_rays, bd, tau, wsum, status, t_n2, t_f2, n2, status2);
        rc = cuda_check(cudaGetLastError(), "tsdf_recovery_bounds launch");
        if (rc) return rc;
    }
    int32_t* sums = reinterpret_cast<int32_t*>((reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255));
    return exclusive_scan(n2, n_rays, offsets2, sums, st);
}

// ---------------------------------------------------------------------------
// tsdf_ray_bounds without a caller workspace.
//
// Some callers cannot allocate device memory of their own: a host application
// that hands the library only buffers it registered at start-up, a real-time
// render loop that forbids any allocation once it runs, or code embedded in a
// framework whose allocator it cannot reach.  For them the only scratch this
// call needs -- the per-chunk partial sums of the offsets scan -- lives in the
// array below, which every device that loads the library holds until exit.
// It is sized for kNoAllocMaxRays rays per call; every call overwrites the
// partial sums it uses before reading them, so nothing has to be cleared, and
// two calls that overlap on the GPU (different streams, no ordering) race on it.
// ---------------------------------------------------------------------------
namespace {
constexpr int64_t kNoAllocMaxRays = (int64_t)1 << 24;
constexpr size_t kNoAllocScratchBytes = (size_t)(((kNoAllocMaxRays + kScanChunk - 1) / kScanChunk) + 1) * sizeof(int32_t) + 256;
static __device__ __align__(256) unsigned char g_bounds_scratch[kNoAllocScratchBytes];

SymbolCache g_scratch_cache;

// device address of g_bounds_scratch in the current context (looked up on the first call
// in each context, so the first call on a device belongs before any stream capture)
int bounds_scratch(void** out) {
    return symbol_address(g_scratch_cache, (const void*)&g_bounds_scratch, out,
                          "tsdf_ray_bounds_noalloc cudaGetSymbolAddress");
}
}  // namespace

extern "C" int64_t tsdf_ray_bounds_noalloc_max_rays(void) { return kNoAllocMaxRays; }

extern "C" int tsdf_ray_bounds_noalloc(const tsdfs_grid* g, const uint32_t* mask, const float* ray_o,
                                       const float* ray_d, int64_t n_rays, const tsdfs_bounds_params* p, float* t_n,
                                       float* t_f, int32_t* n_samples, int32_t* offsets, float* t_zero,
                                       uint8_t* status, tsdfs_stream_t stream) {
    if (n_rays > kNoAllocMaxRays)
        return fail(TSDFS_E_INVALID, "tsdf_ray_bounds_noalloc takes at most %lld rays per call (got %lld); split the batch",
                    (long long)kNoAllocMaxRays, (long long)n_rays);
    void* scratch = nullptr;
    int rc = bounds_scratch(&scratch);
    if (rc) return rc;
    return tsdf_ray_bounds(g, mask, ray_o, ray_d, n_rays, p, t_n, t_f, n_samples, offsets, t_zero, status, scratch,
                           kNoAllocScratchBytes, stream);
}

// ---------------------------------------------------------------------------
// Adaptive sample counts relative to the mean interval (Sec. 3.4: samples at
// equal spacing inside [t_n, t_f], so the count is proportional to the
// interval's length; the supplementary ray study: a ray whose bound is longer
// than the average bound gets more samples, a shorter one fewer).  Two passes:
// the mean length of the BOUNDED intervals over the batch, then per ray
// n = clamp(ceil(L / (mean / n_mean)), n_min, n_max).  The mean is summed in
// FP64 in a fixed order (a fixed grid of kMeanBlocks blocks, each a fixed tree),
// so it does not depend on scheduling, and rounded once to FP32; the count
// arithmetic is FP32 with IEEE division (this file is compiled without FMA
// contraction), so an FP32 restatement on the host reproduces every count.
// ---------------------------------------------------------------------------
namespace tsdfs {
namespace {
constexpr int kMeanBlocks = 256;
constexpr int kMeanThreads = 256;

__global__ void __launch_bounds__(kMeanThreads) k_len_partials(const float* __restrict__ t_n,
                                                                const float* __restrict__ t_f,
                                                                const uint8_t* __restrict__ status, int64_t n_rays,
                                                                double* __restrict__ part_sum,
                                                                unsigned long long* __restrict__ part_cnt) {
    __shared__ double s_sum[kMeanThreads];
    __shared__ unsigned long long s_cnt[kMeanThreads];
    double acc = 0.0;
    unsigned long long cnt = 0;
    for (int64_t r = blockIdx.x * (int64_t)kMeanThreads + threadIdx.x; r < n_rays; r += (int64_t)kMeanBlocks * kMeanThreads) {
        if (__ldg(status + r) == TSDFS_BOUNDED) {
            acc += (double)__fsub_rn(__ldg(t_f + r), __ldg(t_n + r));
            ++cnt;
        }
    }
    s_sum[threadIdx.x] = acc;
    s_cnt[threadIdx.x] = cnt;
    __syncthreads();
    for (int h = kMeanThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s_sum[threadIdx.x] += s_sum[threadIdx.x + h];
            s_cnt[threadIdx.x] += s_cnt[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part_sum[blockIdx.x] = s_sum[0];
        part_cnt[blockIdx.x] = s_cnt[0];
    }
}

// one block: the partials in a fixed tree -> mean (FP32) and the spacing mean / n_mean
__global__ void __launch_bounds__(kMeanBlocks) k_len_mean(const double* __restrict__ part_sum,
                                                          const unsigned long long* __restrict__ part_cnt,
                                                          float n_mean, float* __restrict__ mean_out,
                                                          float* __restrict__ spacing_out) {
    __shared__ double s_sum[kMeanBlocks];
    __shared__ unsigned long long s_cnt[kMeanBlocks];
    s_sum[threadIdx.x] = part_sum[threadIdx.x];
    s_cnt[threadIdx.x] = part_cnt[threadIdx.x];
    __syncthreads();
    for (int h = kMeanBlocks / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s_sum[threadIdx.x] += s_sum[threadIdx.x + h];
            s_cnt[threadIdx.x] += s_cnt[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float mean = s_cnt[0] > 0 ? (float)(s_sum[0] / (double)s_cnt[0]) : 0.0f;
        *spacing_out = __fdiv_rn(mean, n_mean);
        if (mean_out) *mean_out = mean;
    }
}

__global__ void k_adaptive_counts(const float* __restrict__ t_n, const float* __restrict__ t_f,
                                  const uint8_t* __restrict__ status, int64_t n_rays,
                                  const float* __restrict__ spacing, int n_min, int n_max, int n_fallback,
                                  int32_t* __restrict__ n_out) {
    const float dl = __ldg(spacing);
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rays; r += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t st = __ldg(status + r);
        int n = 0;
        if (st == TSDFS_BOUNDED) {
            const float len = __fsub_rn(__ldg(t_f + r), __ldg(t_n + r));
            float q = dl > 0.0f ? ceilf(__fdiv_rn(len, dl)) : (float)n_min;
            q = fminf(fmaxf(q, (float)n_min), (float)n_max);  // also maps NaN to n_min
            n = (int)q;
        } else if (st == TSDFS_FALLBACK) {
            n = n_fallback;
        }
        n_out[r] = n;
    }
}
}  // namespace
}  // namespace tsdfs

extern "C" size_t tsdfs_adaptive_counts_workspace_size(int64_t n_rays) {
    if (n_rays < 0) return 0;
    return tsdfs_bounds_workspace_size(n_rays) + (size_t)kMeanBlocks * (sizeof(double) + sizeof(unsigned long long)) +
           3 * 256;
}

extern "C" int tsdf_adaptive_counts(const float* t_n, const float* t_f, const uint8_t* status, int64_t n_rays,
                                    float n_mean, int32_t n_min, int32_t n_max, int32_t n_fallback,
                                    int32_t* n_samples, int32_t* offsets, float* mean_len, void* ws, size_t ws_bytes,
                                    tsdfs_stream_t stream) {
    if (n_rays < 0 || n_rays > (int64_t)INT32_MAX) return fail(TSDFS_E_INVALID, "n_rays must be in [0, 2^31)");
    if (!(n_mean > 0.0f) || !(n_mean <= 4096.0f)) return fail(TSDFS_E_INVALID, "n_mean must be in (0, 4096]");
    if (n_min < 1 || n_max < n_min || n_max > 4096) return fail(TSDFS_E_INVALID, "need 1 <= n_min <= n_max <= 4096");
    if (n_fallback < 0 || n_fallback > 4096) return fail(TSDFS_E_INVALID, "n_fallback must be in [0, 4096]");
    if ((int64_t)(n_max > n_fallback ? n_max : n_fallback) * n_rays > (int64_t)INT32_MAX)
        return fail(TSDFS_E_INVALID, "sample total could overflow int32 offsets");
    if (n_rays > 0 && (!t_n || !t_f || !status || !n_samples))
        return fail(TSDFS_E_INVALID, "bound, status and count pointers must be non-NULL");
    if (!offsets) return fail(TSDFS_E_INVALID, "offsets is NULL");
    if (!ws || ws_bytes < tsdfs_adaptive_counts_workspace_size(n_rays))
        return fail(TSDFS_E_WORKSPACE, "adaptive counts workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    uintptr_t p = (reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255);
    int32_t* sums = reinterpret_cast<int32_t*>(p);
    p = (p + (size_t)(scan_chunks(n_rays) + 1) * sizeof(int32_t) + 255) & ~uintptr_t(255);
    double* part_sum = reinterpret_cast<double*>(p);
    unsigned long long* part_cnt = reinterpret_cast<unsigned long long*>(p + kMeanBlocks * sizeof(double));
    float* spacing = reinterpret_cast<float*>(p + kMeanBlocks * (sizeof(double) + sizeof(unsigned long long)));
    if (n_rays > 0) {
        ProfScope ps("adaptive_counts", st);
        k_len_partials<<<kMeanBlocks, kMeanThreads, 0, st>>>(t_n, t_f, status, n_rays, part_sum, part_cnt);
        k_len_mean<<<1, kMeanBlocks, 0, st>>>(part_sum, part_cnt, n_mean, mean_len, spacing);
        k_adaptive_counts<<<grid_1d(n_rays, 256), 256, 0, st>>>(t_n, t_f, status, n_rays, spacing, n_min, n_max,
                                                                n_fallback, n_samples);
        int rc = cuda_check(cudaGetLastError(), "adaptive counts launch");
        if (rc) return rc;
    } else if (mean_len) {
        int rc = cuda_check(cudaMemsetAsync(mean_len, 0, sizeof(float), st), "adaptive counts memset");
        if (rc) return rc;
    }
    return exclusive_scan(n_samples, n_rays, offsets, sums, st);
}

// ---------------------------------------------------------------------------
// Autotuner of the march's launch shape.  The march is latency-bound (a DDA per
// thread, scattered reads of an L2-resident grid), so its speed depends on how
// many rays are in flight per SM and how rays are grouped into blocks; the best
// shape depends on the grid, the ray batch and the device.  The candidates are
// every (threads per block, resident blocks per SM) pair below; each is timed
// with CUDA events on the caller's stream over `reps` launches on the caller's
// own rays (outputs are identical for every shape: rays are independent), and
// the fastest becomes this device's shape for tsdf_ray_bounds and
// tsdf_recovery_bounds.  It synchronises the stream: a set-up call.
// ---------------------------------------------------------------------------
namespace {
constexpr int kTuneBlocks[] = {64, 128, 256};
constexpr int kTunePerSm[] = {4, 8, 16, 32, 64};
}  // namespace

extern "C" int tsdfs_bounds_launch_shape(int32_t* block, int32_t* blocks_per_sm) {
    if (!block || !blocks_per_sm) return fail(TSDFS_E_INVALID, "block and blocks_per_sm must be non-NULL");
    const MarchShape sh = march_shape();
    *block = sh.block;
    *blocks_per_sm = sh.blocks_per_sm;
    return TSDFS_OK;
}

extern "C" int tsdfs_set_bounds_launch_shape(int32_t block, int32_t blocks_per_sm) {
    if (block == 0 && blocks_per_sm == 0) {
        block = kBoundsBlock;
        blocks_per_sm = 64;
    }
    if (block < 32 || block > kBoundsMaxBlock || block % 32 != 0 || blocks_per_sm < 1 || blocks_per_sm > 1024)
        return fail(TSDFS_E_INVALID, "block must be a multiple of 32 in [32, %d], blocks_per_sm in [1, 1024]",
                    kBoundsMaxBlock);
    int dev = 0;
    int rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    if (dev < 0 || dev >= 64) return fail(TSDFS_E_UNSUPPORTED, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_shape_mu);
    g_shape[dev].block = block;
    g_shape[dev].blocks_per_sm = blocks_per_sm;
    return TSDFS_OK;
}

extern "C" int tsdfs_autotune_bounds(const tsdfs_grid* g, const uint32_t* mask, const float* ray_o, const float* ray_d,
                                     int64_t n_rays, const tsdfs_bounds_params* p, float* t_n, float* t_f,
                                     int32_t* n_samples, int32_t* offsets, float* t_zero, uint8_t* status, void* ws,
                                     size_t ws_bytes, int32_t reps, float* best_ms, tsdfs_stream_t stream) {
    if (reps < 1 || reps > 1000) return fail(TSDFS_E_INVALID, "reps must be in [1, 1000]");
    if (n_rays < 1) return fail(TSDFS_E_INVALID, "autotuning needs at least one ray");
    int32_t b0 = 0, s0 = 0;
    tsdfs_bounds_launch_shape(&b0, &s0);
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = cuda_check(cudaEventCreate(&e0), "autotune event");
    if (!rc) rc = cuda_check(cudaEventCreate(&e1), "autotune event");
    float best = 1e30f;
    int best_b = b0, best_s = s0;
    for (int bi = 0; !rc && bi < (int)(sizeof(kTuneBlocks) / sizeof(int)); ++bi)
        for (int si = 0; !rc && si < (int)(sizeof(kTunePerSm) / sizeof(int)); ++si) {
            rc = tsdfs_set_bounds_launch_shape(kTuneBlocks[bi], kTunePerSm[si]);
            // one untimed launch (argument checks, caches), then `reps` timed
            if (!rc) rc = tsdf_ray_bounds(g, mask, ray_o, ray_d, n_rays, p, t_n, t_f, n_samples, offsets, t_zero,
                                          status, ws, ws_bytes, stream);
            if (!rc) rc = cuda_check(cudaEventRecord(e0, st), "autotune event record");
            for (int r = 0; !rc && r < reps; ++r)
                rc = tsdf_ray_bounds(g, mask, ray_o, ray_d, n_rays, p, t_n, t_f, n_samples, offsets, t_zero, status,
                                     ws, ws_bytes, stream);
            if (!rc) rc = cuda_check(cudaEventRecord(e1, st), "autotune event record");
            if (!rc) rc = cuda_check(cudaEventSynchronize(e1), "autotune event sync");
            float ms = 0.0f;
            if (!rc) rc = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "autotune elapsed");
            if (!rc && ms < best) {
                best = ms;
                best_b = kTuneBlocks[bi];
                best_s = kTunePerSm[si];
            }
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    const int rc2 = tsdfs_set_bounds_launch_shape(rc ? b0 : best_b, rc ? s0 : best_s);
    if (rc) return rc;
    if (best_ms) *best_ms = best / (float)reps;
    return rc2;
}

// ---------------------------------------------------------------------------
// L2 read-bandwidth probe: the measured peak against which the ray march is
// judged when its grid stays in L2.  Every thread streams 16-byte loads over the
// buffer (which the caller keeps at a size L2 holds) reps times; the XOR of the
// loaded words goes to `sink` so the loads are kept.
// ---------------------------------------------------------------------------
namespace tsdfs {
namespace {
__global__ void k_l2_read(const uint4* __restrict__ buf, int64_t n16, int reps, uint32_t* sink) {
    uint32_t acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r)
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += stride) {
            const uint4 v = __ldcg(buf + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    if (acc == 0x9e3779b9u) *sink = acc;   // practically never taken; keeps the loads live
}
}  // namespace
}  // namespace tsdfs

extern "C" int tsdfs_l2_read_probe(const void* buf, size_t bytes, int32_t reps, uint32_t* sink, float* ms_out,
                                   tsdfs_stream_t stream) {
    using namespace tsdfs;
    if (!buf || !sink || !ms_out || bytes < 16 || reps < 1 || (reinterpret_cast<uintptr_t>(buf) & 15u) != 0)
        return fail(TSDFS_E_INVALID, "tsdfs_l2_read_probe: buf (16-byte aligned), sink, ms_out, bytes >= 16, reps >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t n16 = (int64_t)(bytes / 16);
    const uint4* b = static_cast<const uint4*>(buf);
    // one pass to bring the buffer into L2, then the timed passes
    k_l2_read<<<sms * 4, 512, 0, st>>>(b, n16, 1, sink);
    int rc = cuda_check(cudaGetLastError(), "l2 probe launch");
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rc = cuda_check(cudaEventCreate(&e0), "l2 probe event");
    if (!rc) rc = cuda_check(cudaEventCreate(&e1), "l2 probe event");
    if (!rc) rc = cuda_check(cudaEventRecord(e0, st), "l2 probe record");
    if (!rc) {
        k_l2_read<<<sms * 4, 512, 0, st>>>(b, n16, reps, sink);
        rc = cuda_check(cudaGetLastError(), "l2 probe launch");
    }
    if (!rc) rc = cuda_check(cudaEventRecord(e1, st), "l2 probe record");
    if (!rc) rc = cuda_check(cudaEventSynchronize(e1), "l2 probe sync");
    if (!rc) rc = cuda_check(cudaEventElapsedTime(ms_out, e0, e1), "l2 probe elapsed");
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}
