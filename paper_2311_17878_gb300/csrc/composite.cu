// Volume-rendering compositing (Eq. 1, Eq. 2, the rendered normal) with NeuS
// opacity, and the per-ray steps of the hierarchical comparator (n_c coarse +
// n_f inverse-CDF fine samples; 64 + 32 is the comparator of Tab. 2).
#include "common.cuh"

namespace tsdfs {

namespace {

constexpr int kCompBlock = 128;
constexpr int kMaxCoarse = 64;
constexpr int kMaxFine = 32;
constexpr int kMaxHier = kMaxCoarse + kMaxFine;


// One thread per ray.  Uniform rays: samples offsets[r]..offsets[r+1]; explicit
// rays: r*per_ray .. (r+1)*per_ray.  eik: sum (|grad f| - 1)^2 for BOUNDED rays.
__global__ void __launch_bounds__(kCompBlock) k_composite(const SampleRec* __restrict__ rec,
                                                          const int32_t* __restrict__ offsets, int per_ray,
                                                          const uint8_t* __restrict__ status, int64_t n_rays,
                                                          const int32_t* total_dev, int64_t capacity, Opacity op,
                                                          float* __restrict__ rgb, float* __restrict__ depth,
                                                          float* __restrict__ wsum_out, float* __restrict__ normal,
                                                          float* __restrict__ eik_out, const uint32_t* dev_status) {
    // outputs are zero when the samples overflowed the workspace, and while the device
    // status word holds a timeout of a network kernel (its records may be incomplete)
    const bool overflow = (total_dev && (int64_t)__ldg(total_dev) > capacity) ||
                          (dev_status && (*(const volatile uint32_t*)dev_status & TSDFS_DEV_TIMEOUT));
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
            const float alpha = section_opacity(op, f, dd, dl);
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
                             float* __restrict__ dc, int n_c) {
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
        const float dl = (te - t0) / (float)n_c;
        for (int j = 0; j < n_c; ++j) {
            tc[r * n_c + j] = t0 + ((float)j + 0.5f) * dl;
            dc[r * n_c + j] = dl;
        }
    }
}

// Weight of the section [z0, z1] between two coarse samples from their SDF
// values alone.  NeuS (up-sampling opacity): slope min(own, previous) clipped
// to [-1e3, 0], section ends at mid -/+ slope * dz / 2.  VolSDF: the density
// at the mid value over the section.  T carries the transmittance, prev_slope
// the previous section's slope.
__device__ __forceinline__ float section_weight(float f0, float f1, float z0, float z1, const Opacity& op, float& T,
                                                float& prev_slope) {
    const float dz = z1 - z0;
    const float mid = 0.5f * (f0 + f1);
    const float slope = dz > 0.0f ? (f1 - f0) / dz : 0.0f;
    float c = fminf(slope, prev_slope);
    c = fminf(fmaxf(c, -1e3f), 0.0f);
    prev_slope = slope;
    // the opacity of a section of width dz around the mid value with slope c
    const float alpha = section_opacity(op, mid, c, dz);
    const float w = alpha * T;
    T *= 1.0f - alpha;
    return w;
}

// n_f inverse-CDF samples at u_k = (k + 1/2)/n_f over the c - 1 sections of the
// coarse samples zat(0) < ... < zat(c-1) (c >= 2), pdf ~ w + 1e-5, linear within
// a section.  Two passes over the sections (the normaliser, then the samples
// in increasing u) so that no per-ray table is kept.
template <class Z, class F>
__device__ __forceinline__ void fine_from_coarse(Z zat, F fat, int c, const Opacity& op, int n_f, float* fine) {
    float T = 1.0f, prev_slope = 0.0f, psum = 0.0f;
    for (int j = 0; j < c - 1; ++j)
        psum += section_weight(fat(j), fat(j + 1), zat(j), zat(j + 1), op, T, prev_slope) + 1e-5f;
    const float inv_sum = 1.0f / psum;
    T = 1.0f;
    prev_slope = 0.0f;
    float cum = 0.0f;
    int k = 0;
    for (int j = 0; j < c - 1 && k < n_f; ++j) {
        const float z0 = zat(j), z1 = zat(j + 1);
        const float cnext = cum + (section_weight(fat(j), fat(j + 1), z0, z1, op, T, prev_slope) + 1e-5f);
        const float c0 = cum * inv_sum, c1 = cnext * inv_sum;
        const bool last = j == c - 2;
        while (k < n_f) {
            const float u = ((float)k + 0.5f) / (float)n_f;
            if (!last && c1 <= u) break;
            const float p = c1 - c0;
            fine[k++] = p > 0.0f ? z0 + (u - c0) / p * (z1 - z0) : z0;
        }
        cum = cnext;
    }
}

// Merge the ascending coarse (zat) and fine samples and hand each merged sample
// with its section width (boundaries halfway between sorted neighbours, the
// outer ones at lo and hi) to emit(i, t, delta).
template <class Z, class E>
__device__ __forceinline__ void merge_emit(Z zat, int c, const float* fine, int n_f, float lo, float hi, E emit) {
    const int m = c + n_f;
    int a = 0, b = 0;
    auto pick = [&]() {
        const bool take_c = b >= n_f || (a < c && zat(a) <= fine[b]);
        return take_c ? zat(a++) : fine[b++];
    };
    float prev = 0.0f, cur = m > 0 ? pick() : 0.0f;
    for (int i = 0; i < m; ++i) {
        const float next = i + 1 < m ? pick() : 0.0f;
        const float bl = i == 0 ? lo : 0.5f * (prev + cur);
        const float bh = i == m - 1 ? hi : 0.5f * (cur + next);
        emit(i, cur, bh - bl);
        prev = cur;
        cur = next;
    }
}

// Comparator: n_c coarse values -> n_f fine samples -> n_c + n_f merged samples per ray.
__global__ void k_hier_fine(const float* __restrict__ fcoarse, const float* __restrict__ tc,
                            const float* __restrict__ t0_in, const float* __restrict__ te_in, int64_t n_rays,
                            Opacity op, float* __restrict__ t_out, float* __restrict__ d_out, int n_c, int n_f) {
    const int n_h = n_c + n_f;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rays; r += (int64_t)gridDim.x * blockDim.x) {
        const float* f = fcoarse + r * n_c;
        const float* z = tc + r * n_c;
        auto zat = [&](int j) { return __ldg(z + j); };
        auto fat = [&](int j) { return __ldg(f + j); };
        float fine[kMaxFine];
        fine_from_coarse(zat, fat, n_c, op, n_f, fine);
        float* to = t_out + r * n_h;
        float* dout = d_out + r * n_h;
        merge_emit(zat, n_c, fine, n_f, __ldg(t0_in + r), __ldg(te_in + r), [&](int i, float t, float dl) {
            to[i] = t;
            dout[i] = dl;
        });
    }
}

// Coarse + fine inside the TSDF bound: ray r has c = offsets[r+1] - offsets[r]
// coarse midpoints of [t_n, t_f] (values in fcoarse[offsets[r] ..]); its
// c + n_f merged samples go to offsets2[r] .. with their ray index.  With one
// coarse sample there are no sections: the fine samples are the midpoints of
// n_f equal parts of [t_n, t_f].
__global__ void k_bounded_fine(const float* __restrict__ fcoarse, const int32_t* __restrict__ offsets,
                               const float* __restrict__ t_n, const float* __restrict__ t_f,
                               const int32_t* __restrict__ offsets2, int64_t n_rays, int n_f, Opacity op,
                               int64_t max_coarse, int64_t capacity2, float* __restrict__ t_out,
                               float* __restrict__ d_out, int32_t* __restrict__ ray_out) {
    // over capacity: the network kernels flag it; nothing is written here
    if ((int64_t)__ldg(offsets + n_rays) > max_coarse || (int64_t)__ldg(offsets2 + n_rays) > capacity2) return;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rays; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t base = __ldg(offsets + r);
        const int c = __ldg(offsets + r + 1) - base;
        if (c <= 0) continue;
        const float lo = __ldg(t_n + r), hi = __ldg(t_f + r);
        const float dl = (hi - lo) / (float)c;
        auto zat = [&](int j) { return lo + ((float)j + 0.5f) * dl; };
        auto fat = [&](int j) { return __ldg(fcoarse + base + j); };
        float fine[kMaxFine];
        if (c >= 2) {
            fine_from_coarse(zat, fat, c, op, n_f, fine);
        } else {
            const float df = (hi - lo) / (float)n_f;
            for (int k = 0; k < n_f; ++k) fine[k] = lo + ((float)k + 0.5f) * df;
        }
        const int64_t b2 = __ldg(offsets2 + r);
        merge_emit(zat, c, fine, n_f, lo, hi, [&](int i, float t, float w) {
            t_out[b2 + i] = t;
            d_out[b2 + i] = w;
            ray_out[b2 + i] = (int32_t)r;
        });
    }
}

// merged count per ray: c + n_f for rays with coarse samples, else 0; all 0 when
// the coarse total exceeds max_coarse (the coarse pass flags that overflow)
__global__ void k_bounded_counts(const int32_t* __restrict__ offsets, int64_t n_rays, int n_f, int64_t max_coarse,
                                 int32_t* __restrict__ n2) {
    const bool over = (int64_t)__ldg(offsets + n_rays) > max_coarse;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rays; r += (int64_t)gridDim.x * blockDim.x) {
        const int c = __ldg(offsets + r + 1) - __ldg(offsets + r);
        n2[r] = (!over && c > 0) ? c + n_f : 0;
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
                     const int32_t* total_dev, int64_t capacity, Opacity op, float* rgb, float* depth,
                     float* wsum, float* normal, float* eik, cudaStream_t st) {
    if (n_rays == 0) return TSDFS_OK;
    k_composite<<<grid_1d(n_rays, kCompBlock), kCompBlock, 0, st>>>(rec, offsets, per_ray, status, n_rays, total_dev,
                                                                    capacity, op, rgb, depth, wsum, normal, eik,
                                                                    device_status_word());
    return cuda_check(cudaGetLastError(), "composite launch");
}

int launch_hier_setup(const tsdfs_grid* g, const float* ray_o, const float* ray_d, int64_t n_rays, float t_near,
                      float t_far, float* t0, float* te, uint8_t* status, float* tc, float* dc, int n_c,
                      cudaStream_t st) {
    if (n_c < 2 || n_c > kMaxCoarse) return fail(TSDFS_E_INVALID, "coarse sample count must be in [2, 64]");
    BoxDev box{{g->origin[0], g->origin[1], g->origin[2]}, {g->nx, g->ny, g->nz}, g->voxel_size};
    k_hier_setup<<<grid_1d(n_rays, 128), 128, 0, st>>>(box, ray_o, ray_d, n_rays, t_near, t_far, t0, te, status, tc, dc,
                                                       n_c);
    return cuda_check(cudaGetLastError(), "hier setup launch");
}

int launch_hier_fine(const float* fcoarse, const float* tc, const float* t0, const float* te, int64_t n_rays,
                     Opacity op, float* t_out, float* d_out, int n_c, int n_f, cudaStream_t st) {
    if (n_c < 2 || n_c > kMaxCoarse || n_f < 1 || n_f > kMaxFine)
        return fail(TSDFS_E_INVALID, "sample counts must be coarse in [2, 64], fine in [1, 32]");
    k_hier_fine<<<grid_1d(n_rays, 128), 128, 0, st>>>(fcoarse, tc, t0, te, n_rays, op, t_out, d_out, n_c, n_f);
    return cuda_check(cudaGetLastError(), "hier fine launch");
}

int launch_bounded_counts(const int32_t* offsets, int64_t n_rays, int n_f, int64_t max_coarse, int32_t* n2,
                          cudaStream_t st) {
    k_bounded_counts<<<grid_1d(n_rays, 256), 256, 0, st>>>(offsets, n_rays, n_f, max_coarse, n2);
    return cuda_check(cudaGetLastError(), "bounded counts launch");
}

int launch_bounded_fine(const float* fcoarse, const int32_t* offsets, const float* t_n, const float* t_f,
                        const int32_t* offsets2, int64_t n_rays, int n_f, Opacity op, int64_t max_coarse,
                        int64_t capacity2, float* t_out, float* d_out, int32_t* ray_out, cudaStream_t st) {
    if (n_f < 0 || n_f > kMaxFine) return fail(TSDFS_E_INVALID, "fine sample count must be in [0, 32]");
    k_bounded_fine<<<grid_1d(n_rays, 128), 128, 0, st>>>(fcoarse, offsets, t_n, t_f, offsets2, n_rays, n_f, op,
                                                         max_coarse, capacity2, t_out, d_out, ray_out);
    return cuda_check(cudaGetLastError(), "bounded fine launch");
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
