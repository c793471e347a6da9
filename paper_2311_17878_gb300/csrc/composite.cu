// Volume-rendering compositing (Eq. 1, Eq. 2, the rendered normal) with NeuS
// opacity, and the per-ray steps of the 64 + 32 hierarchical comparator.
#include "common.cuh"

namespace tsdfs {

namespace {

constexpr int kCompBlock = 128;
constexpr int kCoarse = 64;
constexpr int kFine = 32;
constexpr int kHier = kCoarse + kFine;

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }

// One thread per ray.  Uniform rays: samples offsets[r]..offsets[r+1]; explicit
// rays: r*per_ray .. (r+1)*per_ray.  eik: sum (|grad f| - 1)^2 for BOUNDED rays.
__global__ void __launch_bounds__(kCompBlock) k_composite(const SampleRec* __restrict__ rec,
                                                          const int32_t* __restrict__ offsets, int per_ray,
                                                          const uint8_t* __restrict__ status, int64_t n_rays,
                                                          const int32_t* total_dev, int64_t capacity, float inv_s,
                                                          float eps, float* __restrict__ rgb, float* __restrict__ depth,
                                                          float* __restrict__ wsum_out, float* __restrict__ normal,
                                                          float* __restrict__ eik_out) {
    const bool overflow = total_dev && (int64_t)__ldg(total_dev) > capacity;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rays; r += (int64_t)gridDim.x * blockDim.x) {
        int64_t b, e;
        if (offsets) {
            b = __ldg(offsets + r);
            e = __ldg(offsets + r + 1);
        } else {
            b = r * per_ray;
            e = b + per_ray;
        }
        const uint8_t st = status ? __ldg(status + r) : (uint8_t)TSDFS_BOUNDED;
        if (overflow || st == TSDFS_MISS) e = b;
        float logT = 0.0f, ws = 0.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f, dt = 0.0f, nx = 0.0f, ny = 0.0f, nz = 0.0f;
        float eik = 0.0f;
        for (int64_t g = b; g < e; ++g) {
            const float4 q0 = reinterpret_cast<const float4*>(rec + g)[0];
            const float4 q1 = reinterpret_cast<const float4*>(rec + g)[1];
            const float4 q2 = reinterpret_cast<const float4*>(rec + g)[2];
            const float f = q0.x, dd = q0.y, t = q0.z, dl = q0.w;
            const float c = fminf(dd, 0.0f);
            const float p_lo = sigmoidf_(inv_s * (f - 0.5f * dl * c));
            const float p_hi = sigmoidf_(inv_s * (f + 0.5f * dl * c));
            float alpha = (p_lo - p_hi + eps) / (p_lo + eps);
            alpha = fminf(fmaxf(alpha, 0.0f), 1.0f);
            const float w = expf(logT) * alpha;
            ws += w;
            cr += w * q1.x; cg += w * q1.y; cb += w * q1.z;
            dt += w * t;
            nx += w * q2.x; ny += w * q2.y; nz += w * q2.z;
            const float gm = q1.w - 1.0f;
            eik += gm * gm;
            logT += log1pf(-fminf(alpha, 1.0f - 5.9604645e-8f));
        }
        const bool ok = ws >= 1e-8f;
        const float inv = ok ? 1.0f / ws : 0.0f;
        rgb[3 * r + 0] = cr; rgb[3 * r + 1] = cg; rgb[3 * r + 2] = cb;
        depth[r] = ok ? dt * inv : 0.0f;
        wsum_out[r] = ws;
        if (normal) {
            normal[3 * r + 0] = ok ? nx * inv : 0.0f;
            normal[3 * r + 1] = ok ? ny * inv : 0.0f;
            normal[3 * r + 2] = ok ? nz * inv : 0.0f;
        }
        if (eik_out) eik_out[r] = st == TSDFS_BOUNDED && !overflow ? eik : 0.0f;
    }
}

// [t0, t_end] of each ray against the grid box (same slab test as the bounds kernel)
__device__ __forceinline__ bool clip_box(const float o[3], const float d[3], const float org[3], const int n[3], float vs,
                                         float t_near, float t_far, float& t0, float& t_end) {
    const float kInf = __int_as_float(0x7f800000);
    float tmin = -kInf, tmax = kInf;
    bool hit = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = org[a], hi = __fadd_rn(org[a], __fmul_rn((float)n[a], vs));
        if (d[a] == 0.0f) {
            if (o[a] < lo || o[a] > hi) hit = false;
            continue;
        }
        const float inv = __fdiv_rn(1.0f, d[a]);
        const float t1 = __fmul_rn(__fsub_rn(lo, o[a]), inv), t2 = __fmul_rn(__fsub_rn(hi, o[a]), inv);
        const float tl = t1 < t2 ? t1 : t2, th = t1 < t2 ? t2 : t1;
        if (tl > tmin) tmin = tl;
        if (th < tmax) tmax = th;
    }
    t0 = t_near > tmin ? t_near : tmin;
    t_end = t_far < tmax ? t_far : tmax;
    return hit && t0 < t_end;
}

struct BoxDev {
    float org[3];
    int n[3];
    float vs;
};

__global__ void k_hier_setup(BoxDev box, const float* __restrict__ ray_o, const float* __restrict__ ray_d,
                             int64_t n_rays, float t_near, float t_far, float* __restrict__ t0_out,
                             float* __restrict__ te_out, uint8_t* __restrict__ status, float* __restrict__ tc,
                             float* __restrict__ dc) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rays; r += (int64_t)gridDim.x * blockDim.x) {
        float o[3], d[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = __ldg(ray_o + 3 * r + a);
            d[a] = __ldg(ray_d + 3 * r + a);
        }
        float t0, te;
        const bool ok = clip_box(o, d, box.org, box.n, box.vs, t_near, t_far, t0, te);
        if (!ok) { t0 = 0.0f; te = 0.0f; }
        t0_out[r] = t0;
        te_out[r] = te;
        status[r] = ok ? TSDFS_FALLBACK : TSDFS_MISS;
        const float dl = (te - t0) / (float)kCoarse;
        for (int j = 0; j < kCoarse; ++j) {
            tc[r * kCoarse + j] = t0 + ((float)j + 0.5f) * dl;
            dc[r * kCoarse + j] = dl;
        }
    }
}

// Section weights from the coarse SDF values, 32 inverse-CDF samples, merge,
// and section widths with boundaries halfway between sorted neighbours.
__global__ void k_hier_fine(const float* __restrict__ fcoarse, const float* __restrict__ tc,
                            const float* __restrict__ t0_in, const float* __restrict__ te_in, int64_t n_rays,
                            float inv_s, float eps, float* __restrict__ t_out, float* __restrict__ d_out) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rays; r += (int64_t)gridDim.x * blockDim.x) {
        const float* f = fcoarse + r * kCoarse;
        const float* z = tc + r * kCoarse;
        float cdf[kCoarse];
        // section weights w_j (j < 63) -> pdf ~ w + 1e-5 -> cdf[0..63]
        float T = 1.0f, prev_slope = 0.0f, psum = 0.0f;
        cdf[0] = 0.0f;
        for (int j = 0; j < kCoarse - 1; ++j) {
            const float f0 = __ldg(f + j), f1 = __ldg(f + j + 1);
            const float z0 = __ldg(z + j), z1 = __ldg(z + j + 1);
            const float dz = z1 - z0;
            const float mid = 0.5f * (f0 + f1);
            const float slope = dz > 0.0f ? (f1 - f0) / dz : 0.0f;
            float c = fminf(slope, prev_slope);
            c = fminf(fmaxf(c, -1e3f), 0.0f);
            prev_slope = slope;
            const float p_lo = sigmoidf_(inv_s * (mid - 0.5f * c * dz));
            const float p_hi = sigmoidf_(inv_s * (mid + 0.5f * c * dz));
            float alpha = (p_lo - p_hi + eps) / (p_lo + eps);
            alpha = fminf(fmaxf(alpha, 0.0f), 1.0f);
            const float w = alpha * T;
            T *= 1.0f - alpha;
            psum += w + 1e-5f;
            cdf[j + 1] = psum;
        }
        const float inv_sum = 1.0f / psum;
        // inverse CDF at u_k = (k + 1/2)/32 (u increasing -> samples increasing)
        float fine[kFine];
        int j = 0;
        for (int k = 0; k < kFine; ++k) {
            const float u = ((float)k + 0.5f) / (float)kFine;
            while (j < kCoarse - 2 && cdf[j + 1] * inv_sum <= u) ++j;
            const float c0 = cdf[j] * inv_sum, c1 = cdf[j + 1] * inv_sum;
            const float p = c1 - c0;
            const float z0 = __ldg(z + j), z1 = __ldg(z + j + 1);
            fine[k] = p > 0.0f ? z0 + (u - c0) / p * (z1 - z0) : z0;
        }
        // merge 64 coarse + 32 fine (both ascending)
        float ts[kHier];
        int a = 0, b = 0;
        for (int i = 0; i < kHier; ++i) {
            const bool take_c = b >= kFine || (a < kCoarse && __ldg(z + a) <= fine[b]);
            ts[i] = take_c ? __ldg(z + a++) : fine[b++];
        }
        const float lo = __ldg(t0_in + r), hi = __ldg(te_in + r);
        for (int i = 0; i < kHier; ++i) {
            const float bl = i == 0 ? lo : 0.5f * (ts[i - 1] + ts[i]);
            const float bh = i == kHier - 1 ? hi : 0.5f * (ts[i] + ts[i + 1]);
            t_out[r * kHier + i] = ts[i];
            d_out[r * kHier + i] = bh - bl;
        }
    }
}

// recovery merge: rays re-rendered by the recovery pass take the second render's outputs
__global__ void k_recovery_merge(int64_t n_rays, const uint8_t* __restrict__ status2, const float* __restrict__ rgb2,
                                 const float* __restrict__ depth2, const float* __restrict__ wsum2,
                                 const float* __restrict__ normal2, float* __restrict__ rgb, float* __restrict__ depth,
                                 float* __restrict__ wsum, float* __restrict__ normal) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rays; r += (int64_t)gridDim.x * blockDim.x) {
        if (status2[r] != TSDFS_FALLBACK) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c) rgb[3 * r + c] = rgb2[3 * r + c];
        depth[r] = depth2[r];
        wsum[r] = wsum2[r];
        if (normal && normal2) {
#pragma unroll
            for (int c = 0; c < 3; ++c) normal[3 * r + c] = normal2[3 * r + c];
        }
    }
}

}  // namespace

int launch_composite(const SampleRec* rec, const int32_t* offsets, int per_ray, const uint8_t* status, int64_t n_rays,
                     const int32_t* total_dev, int64_t capacity, float inv_s, float eps, float* rgb, float* depth,
                     float* wsum, float* normal, float* eik, cudaStream_t st) {
    if (n_rays == 0) return TSDFS_OK;
    k_composite<<<grid_1d(n_rays, kCompBlock), kCompBlock, 0, st>>>(rec, offsets, per_ray, status, n_rays, total_dev,
                                                                    capacity, inv_s, eps, rgb, depth, wsum, normal, eik);
    return cuda_check(cudaGetLastError(), "composite launch");
}

int launch_hier_setup(const tsdfs_grid* g, const float* ray_o, const float* ray_d, int64_t n_rays, float t_near,
                      float t_far, float* t0, float* te, uint8_t* status, float* tc, float* dc, cudaStream_t st) {
    BoxDev box{{g->origin[0], g->origin[1], g->origin[2]}, {g->nx, g->ny, g->nz}, g->voxel_size};
    k_hier_setup<<<grid_1d(n_rays, 128), 128, 0, st>>>(box, ray_o, ray_d, n_rays, t_near, t_far, t0, te, status, tc, dc);
    return cuda_check(cudaGetLastError(), "hier setup launch");
}

int launch_hier_fine(const float* fcoarse, const float* tc, const float* t0, const float* te, int64_t n_rays,
                     float inv_s, float eps, float* t_out, float* d_out, cudaStream_t st) {
    k_hier_fine<<<grid_1d(n_rays, 128), 128, 0, st>>>(fcoarse, tc, t0, te, n_rays, inv_s, eps, t_out, d_out);
    return cuda_check(cudaGetLastError(), "hier fine launch");
}

}  // namespace tsdfs

using namespace tsdfs;

extern "C" int tsdf_recovery_merge(int64_t n_rays, const uint8_t* status2, const float* rgb2, const float* depth2,
                                   const float* wsum2, const float* normal2, float* rgb, float* depth, float* wsum,
                                   float* normal, tsdfs_stream_t stream) {
    if (n_rays < 0) return fail(TSDFS_E_INVALID, "n_rays must be >= 0");
    if (n_rays == 0) return TSDFS_OK;
    if (!status2 || !rgb2 || !depth2 || !wsum2 || !rgb || !depth || !wsum)
        return fail(TSDFS_E_INVALID, "status, colour, depth and weight pointers must be non-NULL");
    if ((normal == nullptr) != (normal2 == nullptr)) return fail(TSDFS_E_INVALID, "normal and normal2: both or neither");
    cudaStream_t st = (cudaStream_t)stream;
    ProfScope ps("recovery_merge", st);
    k_recovery_merge<<<grid_1d(n_rays, 256), 256, 0, st>>>(n_rays, status2, rgb2, depth2, wsum2, normal2, rgb, depth,
                                                          wsum, normal);
    return cuda_check(cudaGetLastError(), "tsdf_recovery_merge launch");
}
