// K1: projective TSDF fusion (Sec. 3.2, Eq. 3, Alg. 2 in its per-voxel form)
// K2: the far-phase neighbourhood test of Alg. 1 as a bit mask.
//
// K1 arithmetic is IEEE fp32 round-to-nearest with no contraction (explicit
// __f*_rn intrinsics, and this file is compiled with --fmad=false), in the
// operation order that tsdfs.h documents, so pixel choices, weights and
// values are reproducible bit for bit.
#include "common.cuh"
#include "march.cuh"

namespace tsdfs {

namespace {

constexpr int kFuseBlock = 256;

__device__ __forceinline__ float load_v(const void* V, int f16, int64_t idx) {
    return f16 ? __half2float(reinterpret_cast<const __half*>(V)[idx]) : reinterpret_cast<const float*>(V)[idx];
}
__device__ __forceinline__ void store_v(void* V, int f16, int64_t idx, float v) {
    if (f16) reinterpret_cast<__half*>(V)[idx] = __float2half_rn(v);
    else reinterpret_cast<float*>(V)[idx] = v;
}

__global__ void k_grid_init(void* V, int f16, uint8_t* W, int64_t n) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        store_v(V, f16, q, -1.0f);
        W[q] = 0;
    }
}

// One thread per voxel; the camera table of all views is staged in shared
// memory (16 floats per view: c2w[12], fx, fy, cx, cy).
__global__ void __launch_bounds__(kFuseBlock) k_integrate(int nx, int ny, int nz, float ox, float oy, float oz,
                                                          float vs, float trunc, void* V, int f16, uint8_t* W,
                                                          const float* __restrict__ depth, int nv, int H, int Wd,
                                                          const float* __restrict__ Kc, const float* __restrict__ c2w) {
    extern __shared__ float cam[];
    for (int i = threadIdx.x; i < nv * 16; i += blockDim.x) {
        int v = i >> 4, c = i & 15;
        cam[i] = c < 12 ? c2w[v * 12 + c] : Kc[v * 4 + (c - 12)];
    }
    __syncthreads();
    const int64_t n = (int64_t)nx * ny * nz;
    const float fW = (float)Wd, fH = (float)H;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % nx);
        const int j = (int)((q / nx) % ny);
        const int k = (int)(q / ((int64_t)nx * ny));
        const float cx = __fadd_rn(ox, __fmul_rn(__fadd_rn((float)i, 0.5f), vs));
        const float cy = __fadd_rn(oy, __fmul_rn(__fadd_rn((float)j, 0.5f), vs));
        const float cz = __fadd_rn(oz, __fmul_rn(__fadd_rn((float)k, 0.5f), vs));
        float Vv = load_v(V, f16, q);
        int Wv = W[q];
        for (int view = 0; view < nv; ++view) {
            const float* P = cam + view * 16;
            const float dx = __fsub_rn(cx, P[3]), dy = __fsub_rn(cy, P[7]), dz = __fsub_rn(cz, P[11]);
            const float zc = __fadd_rn(__fadd_rn(__fmul_rn(P[2], dx), __fmul_rn(P[6], dy)), __fmul_rn(P[10], dz));
            if (!(zc > 0.0f)) continue;
            const float xc = __fadd_rn(__fadd_rn(__fmul_rn(P[0], dx), __fmul_rn(P[4], dy)), __fmul_rn(P[8], dz));
            const float yc = __fadd_rn(__fadd_rn(__fmul_rn(P[1], dx), __fmul_rn(P[5], dy)), __fmul_rn(P[9], dz));
            const float fx = P[12], fy = P[13], ccx = P[14], ccy = P[15];
            const float u = __fadd_rn(__fmul_rn(fx, __fdiv_rn(xc, zc)), ccx);
            const float v = __fadd_rn(__fmul_rn(fy, __fdiv_rn(yc, zc)), ccy);
            if (!(u >= 0.0f && u < fW && v >= 0.0f && v < fH)) continue;
            int px = (int)floorf(u), py = (int)floorf(v);
            px = px >= Wd ? Wd - 1 : px;
            py = py >= H ? H - 1 : py;
            const float D = __ldg(depth + ((int64_t)view * H + py) * Wd + px);
            const float a = __fdiv_rn(__fsub_rn(__fadd_rn((float)px, 0.5f), ccx), fx);
            const float b = __fdiv_rn(__fsub_rn(__fadd_rn((float)py, 0.5f), ccy), fy);
            const float nrm = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b)), 1.0f));
            const float proj = __fdiv_rn(__fadd_rn(__fadd_rn(__fmul_rn(a, xc), __fmul_rn(b, yc)), zc), nrm);
            float s = __fsub_rn(D, proj);
            if (s > trunc) s = trunc;
            if (s < -trunc) s = -trunc;
            if (s > -trunc) {
                const float sn = __fdiv_rn(s, trunc);
                const float Wf = (float)Wv;
                Vv = __fdiv_rn(__fadd_rn(__fmul_rn(Wf, Vv), sn), __fadd_rn(Wf, 1.0f));
                if (Wv < 255) ++Wv;
            }
        }
        store_v(V, f16, q, Vv);
        W[q] = (uint8_t)Wv;
    }
}

// K2: inside bit of voxel X = all voxels within Chebyshev radius r have V < 0,
// computed as a separable running maximum over a shared-memory halo tile.
constexpr int kMTX = 32, kMTY = 4, kMTZ = 4, kMaxR = 4;

__global__ void __launch_bounds__(kMTX * kMTY) k_inside_mask(const void* __restrict__ V, int f16, int nx, int ny,
                                                             int nz, int r, uint32_t* __restrict__ bits,
                                                             int aligned_rows) {
    constexpr int HX = kMTX + 2 * kMaxR, HY = kMTY + 2 * kMaxR, HZ = kMTZ + 2 * kMaxR;
    __shared__ float a[HZ][HY][HX];
    __shared__ float bx[HZ][HY][kMTX];
    __shared__ float by[HZ][kMTY][kMTX];
    const int x0 = blockIdx.x * kMTX, y0 = blockIdx.y * kMTY, z0 = blockIdx.z * kMTZ;
    const int hx = kMTX + 2 * r, hy = kMTY + 2 * r, hz = kMTZ + 2 * r;
    const int tid = threadIdx.x + threadIdx.y * kMTX;
    const int nthr = kMTX * kMTY;
    for (int e = tid; e < hx * hy * hz; e += nthr) {
        int lx = e % hx, ly = (e / hx) % hy, lz = e / (hx * hy);
        int gx = x0 + lx - r, gy = y0 + ly - r, gz = z0 + lz - r;
        float v = -1.0f;  // out of grid = unseen
        if (gx >= 0 && gy >= 0 && gz >= 0 && gx < nx && gy < ny && gz < nz) v = load_v(V, f16, ((int64_t)gz * ny + gy) * nx + gx);
        a[lz][ly][lx] = v;
    }
    __syncthreads();
    for (int e = tid; e < kMTX * hy * hz; e += nthr) {
        int lx = e % kMTX, ly = (e / kMTX) % hy, lz = e / (kMTX * hy);
        float m = a[lz][ly][lx];
        for (int d = 1; d <= 2 * r; ++d) m = fmaxf(m, a[lz][ly][lx + d]);
        bx[lz][ly][lx] = m;
    }
    __syncthreads();
    for (int e = tid; e < kMTX * kMTY * hz; e += nthr) {
        int lx = e % kMTX, ly = (e / kMTX) % kMTY, lz = e / (kMTX * kMTY);
        float m = bx[lz][ly][lx];
        for (int d = 1; d <= 2 * r; ++d) m = fmaxf(m, bx[lz][ly + d][lx]);
        by[lz][ly][lx] = m;
    }
    __syncthreads();
    const int lx = threadIdx.x, ly = threadIdx.y;
    for (int lz = 0; lz < kMTZ; ++lz) {
        float m = by[lz][ly][lx];
        for (int d = 1; d <= 2 * r; ++d) m = fmaxf(m, by[lz + d][ly][lx]);
        const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
        const bool valid = gx < nx && gy < ny && gz < nz;
        const bool inside = valid && m < 0.0f;
        const int64_t idx = ((int64_t)gz * ny + gy) * nx + gx;
        if (aligned_rows) {
            unsigned word = __ballot_sync(0xffffffffu, inside);
            if (lx == 0 && gy < ny && gz < nz) bits[idx >> 5] = word;
        } else if (inside) {
            atomicOr(bits + (idx >> 5), 1u << (idx & 31));
        }
    }
}

// ---- Alg. 2 as printed, one view at a time: march every pixel's ray ---------------
// Thread per pixel of view `view`: unit ray through the pixel centre, clipped to the grid
// box from t = 0; voxel walk of Alg. 1; at each voxel s = clamp(v . (p* - c), -D_T, D_T),
// p* = o + D v (D = +inf: s = D_T); stop at the first s <= -D_T, else add s / D_T in fixed
// point (2^-32 units: integer sums, so the result does not depend on the order in which
// the rays arrive) and one count to the voxel.  k_raycast_apply folds the view's sums in.
constexpr double kFix = 4294967296.0;   // 2^32

__global__ void __launch_bounds__(kFuseBlock) k_raycast_view(GridDev g, const float* __restrict__ depth, int H, int Wd,
                                                             const float* __restrict__ Kc, const float* __restrict__ c2w,
                                                             int view, unsigned long long* __restrict__ qsum,
                                                             uint32_t* __restrict__ cnt) {
    const float kInf = __int_as_float(0x7f800000);
    const float* P = c2w + 12 * view;
    const float fx = __ldg(Kc + 4 * view), fy = __ldg(Kc + 4 * view + 1);
    const float cx = __ldg(Kc + 4 * view + 2), cy = __ldg(Kc + 4 * view + 3);
    const float o[3] = {__ldg(P + 3), __ldg(P + 7), __ldg(P + 11)};
    const int max_steps = g.n[0] + g.n[1] + g.n[2] + 8;
    const int64_t n_pix = (int64_t)H * Wd;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_pix; q += (int64_t)gridDim.x * blockDim.x) {
        const int px = (int)(q % Wd), py = (int)(q / Wd);
        const float a = __fdiv_rn(__fsub_rn(__fadd_rn((float)px, 0.5f), cx), fx);
        const float b = __fdiv_rn(__fsub_rn(__fadd_rn((float)py, 0.5f), cy), fy);
        float d[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            d[k] = __fadd_rn(__fadd_rn(__fmul_rn(__ldg(P + 4 * k), a), __fmul_rn(__ldg(P + 4 * k + 1), b)),
                             __ldg(P + 4 * k + 2));
        const float nn = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(d[0], d[0]), __fmul_rn(d[1], d[1])), __fmul_rn(d[2], d[2])));
#pragma unroll
        for (int k = 0; k < 3; ++k) d[k] = __fdiv_rn(d[k], nn);
        const float D = __ldg(depth + ((int64_t)view * H + py) * Wd + px);
        float t0, t_end;
        if (!clip_box(g, o, d, 0.0f, kInf, t0, t_end)) continue;
        float ps[3];   // p* = o + D v
#pragma unroll
        for (int k = 0; k < 3; ++k) ps[k] = __fadd_rn(o[k], __fmul_rn(D, d[k]));
        const bool free_ray = isinf(D);
        Dda s;
        dda_init(s, g, o, d, t0);
        for (int st = 0; st < max_steps && s.t < t_end; ++st) {
            float sx = g.trunc;
            if (!free_ray) {
                float e[3];
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    e[k] = __fsub_rn(ps[k], __fadd_rn(g.org[k], __fmul_rn(__fadd_rn((float)s.X[k], 0.5f), g.vs)));
                const float dot = __fadd_rn(__fadd_rn(__fmul_rn(d[0], e[0]), __fmul_rn(d[1], e[1])), __fmul_rn(d[2], e[2]));
                sx = dot > g.trunc ? g.trunc : (dot < -g.trunc ? -g.trunc : dot);
            }
            if (!(sx > -g.trunc)) break;
            const long long qv = __double2ll_rn((double)__fdiv_rn(sx, g.trunc) * kFix);
            const int64_t idx = ((int64_t)s.X[2] * g.n[1] + s.X[1]) * g.n[0] + s.X[0];
            atomicAdd(qsum + idx, (unsigned long long)qv);
            atomicAdd(cnt + idx, 1u);
            if (!dda_next(s, g, o)) break;
        }
    }
}

// the view's k visits of a voxel: V <- (W V + sum) / (W + k) in FP64, rounded once to the
// storage type; W <- min(W + k, 255); the accumulators are cleared for the next view
__global__ void k_raycast_apply(void* V, int f16, uint8_t* W, unsigned long long* __restrict__ qsum,
                                uint32_t* __restrict__ cnt, int64_t n) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = cnt[q];
        if (k == 0) continue;
        const long long sum = (long long)qsum[q];
        const float v = load_v(V, f16, q);
        const uint32_t w = W[q];
        const double vn = ((double)w * (double)v + (double)sum / kFix) / (double)(w + k);
        store_v(V, f16, q, (float)vn);
        W[q] = (uint8_t)(w + k > 255u ? 255u : w + k);
        qsum[q] = 0ull;
        cnt[q] = 0u;
    }
}

}  // namespace

int grid_check(const tsdfs_grid* g) {
    if (!g) return fail(TSDFS_E_INVALID, "grid is NULL");
    if (g->nx <= 0 || g->ny <= 0 || g->nz <= 0) return fail(TSDFS_E_INVALID, "grid dimensions must be positive");
    if ((int64_t)g->nx * g->ny * g->nz > ((int64_t)1 << 40)) return fail(TSDFS_E_INVALID, "grid too large");
    if (!(g->voxel_size > 0.0f) || !(g->trunc > 0.0f)) return fail(TSDFS_E_INVALID, "voxel_size and trunc must be > 0");
    if (g->dtype != TSDFS_F32 && g->dtype != TSDFS_F16) return fail(TSDFS_E_INVALID, "grid dtype must be TSDFS_F32 or TSDFS_F16");
    if (!g->tsdf) return fail(TSDFS_E_INVALID, "grid tsdf pointer is NULL");
    return TSDFS_OK;
}

}  // namespace tsdfs

using namespace tsdfs;

extern "C" int tsdfs_grid_init(const tsdfs_grid* g, tsdfs_stream_t stream) {
    int rc = grid_check(g);
    if (rc) return rc;
    if (!g->weight) return fail(TSDFS_E_INVALID, "grid weight pointer is NULL");
    int64_t n = (int64_t)g->nx * g->ny * g->nz;
    k_grid_init<<<grid_1d(n, 256), 256, 0, (cudaStream_t)stream>>>(g->tsdf, g->dtype == TSDFS_F16, g->weight, n);
    return cuda_check(cudaGetLastError(), "tsdfs_grid_init launch");
}

extern "C" int tsdf_integrate(const tsdfs_grid* g, const float* depth, int32_t n_views, int32_t H, int32_t W,
                              const float* K, const float* c2w, tsdfs_stream_t stream) {
    int rc = grid_check(g);
    if (rc) return rc;
    if (!g->weight) return fail(TSDFS_E_INVALID, "grid weight pointer is NULL");
    if (n_views < 0 || H <= 0 || W <= 0) return fail(TSDFS_E_INVALID, "n_views must be >= 0 and H, W > 0");
    if (n_views == 0) return TSDFS_OK;
    if (n_views > 2048) return fail(TSDFS_E_INVALID, "at most 2048 views per call (split larger sets)");
    if (!depth || !K || !c2w) return fail(TSDFS_E_INVALID, "depth, K and c2w must be non-NULL");
    int64_t n = (int64_t)g->nx * g->ny * g->nz;
    size_t smem = (size_t)n_views * 16 * sizeof(float);
    if (smem > 48 * 1024) {
        rc = cuda_check(cudaFuncSetAttribute(k_integrate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                        "tsdf_integrate smem attribute");
        if (rc) return rc;
    }
    ProfScope ps("integrate", (cudaStream_t)stream);
    k_integrate<<<grid_1d(n, kFuseBlock, 152 * 8), kFuseBlock, smem, (cudaStream_t)stream>>>(
        g->nx, g->ny, g->nz, g->origin[0], g->origin[1], g->origin[2], g->voxel_size, g->trunc, g->tsdf,
        g->dtype == TSDFS_F16, g->weight, depth, n_views, H, W, K, c2w);
    return cuda_check(cudaGetLastError(), "tsdf_integrate launch");
}

extern "C" size_t tsdfs_raycast_workspace_size(const tsdfs_grid* g) {
    if (!g || g->nx <= 0 || g->ny <= 0 || g->nz <= 0) return 0;
    const int64_t n = (int64_t)g->nx * g->ny * g->nz;
    return (size_t)n * (sizeof(unsigned long long) + sizeof(uint32_t)) + 512;
}

extern "C" int tsdf_integrate_raycast(const tsdfs_grid* g, const float* depth, int32_t n_views, int32_t H, int32_t W,
                                      const float* K, const float* c2w, void* ws, size_t ws_bytes,
                                      tsdfs_stream_t stream) {
    int rc = grid_check(g);
    if (rc) return rc;
    if (!g->weight) return fail(TSDFS_E_INVALID, "grid weight pointer is NULL");
    if (n_views < 0 || H <= 0 || W <= 0) return fail(TSDFS_E_INVALID, "n_views must be >= 0 and H, W > 0");
    if (n_views == 0) return TSDFS_OK;
    if (!depth || !K || !c2w) return fail(TSDFS_E_INVALID, "depth, K and c2w must be non-NULL");
    if ((int64_t)H * W > (int64_t)1 << 21)
        return fail(TSDFS_E_INVALID, "at most 2^21 pixels per view (the fixed-point sums hold 2^21 visits)");
    if (!ws || ws_bytes < tsdfs_raycast_workspace_size(g)) return fail(TSDFS_E_WORKSPACE, "raycast workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = (int64_t)g->nx * g->ny * g->nz;
    uintptr_t p = (reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255);
    unsigned long long* qsum = reinterpret_cast<unsigned long long*>(p);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(p + (size_t)n * sizeof(unsigned long long));
    ProfScope ps("integrate_raycast", st);
    rc = cuda_check(cudaMemsetAsync(qsum, 0, (size_t)n * (sizeof(unsigned long long) + sizeof(uint32_t)), st),
                    "raycast workspace clear");
    if (rc) return rc;
    GridDev gd{g->tsdf, g->dtype == TSDFS_F16, {g->nx, g->ny, g->nz}, {g->origin[0], g->origin[1], g->origin[2]},
               g->voxel_size, g->trunc};
    const int f16 = g->dtype == TSDFS_F16;
    for (int v = 0; v < n_views; ++v) {
        k_raycast_view<<<grid_1d((int64_t)H * W, kFuseBlock, 152 * 16), kFuseBlock, 0, st>>>(gd, depth, H, W, K, c2w, v,
                                                                                            qsum, cnt);
        k_raycast_apply<<<grid_1d(n, 256, 152 * 16), 256, 0, st>>>(g->tsdf, f16, g->weight, qsum, cnt, n);
    }
    return cuda_check(cudaGetLastError(), "tsdf_integrate_raycast launch");
}

extern "C" int64_t tsdfs_inside_mask_words(const tsdfs_grid* g) {
    if (!g || g->nx <= 0 || g->ny <= 0 || g->nz <= 0) return 0;
    return ((int64_t)g->nx * g->ny * g->nz + 31) / 32;
}

extern "C" int tsdfs_inside_mask(const tsdfs_grid* g, int32_t r, uint32_t* bits, tsdfs_stream_t stream) {
    int rc = grid_check(g);
    if (rc) return rc;
    if (r < 0 || r > kMaxR) return fail(TSDFS_E_INVALID, "nb_radius must be in [0, %d]", kMaxR);
    if (!bits) return fail(TSDFS_E_INVALID, "mask_bits is NULL");
    int aligned = (g->nx % 32) == 0;
    if (!aligned) {
        rc = cuda_check(cudaMemsetAsync(bits, 0, (size_t)tsdfs_inside_mask_words(g) * 4, (cudaStream_t)stream),
                        "tsdfs_inside_mask memset");
        if (rc) return rc;
    }
    dim3 grid((g->nx + kMTX - 1) / kMTX, (g->ny + kMTY - 1) / kMTY, (g->nz + kMTZ - 1) / kMTZ);
    if (grid.y > 65535 || grid.z > 65535) return fail(TSDFS_E_INVALID, "grid too large for the mask kernel");
    ProfScope ps("inside_mask", (cudaStream_t)stream);
    k_inside_mask<<<grid, dim3(kMTX, kMTY), 0, (cudaStream_t)stream>>>(g->tsdf, g->dtype == TSDFS_F16, g->nx, g->ny,
                                                                       g->nz, r, bits, aligned);
    return cuda_check(cudaGetLastError(), "tsdfs_inside_mask launch");
}
