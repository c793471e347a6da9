// The voxel walk of Alg. 1 / Alg. 2 ("NextVoxel") and the grid-box clip, shared by the
// ray march (bounds.cu) and the ray-casting fusion (integrate.cu).  Every operation is an
// explicitly rounded IEEE binary32 operation (no contraction), so the walk is the same
// voxel sequence wherever it runs.
#pragma once
#include <cuda_fp16.h>

#include "common.cuh"

namespace tsdfs {
namespace {

struct GridDev {
    const void* V;
    int f16;
    int n[3];
    float org[3];
    float vs;
    float trunc;
};

__device__ __forceinline__ float gval(const GridDev& g, int i, int j, int k) {
    if (i < 0 || j < 0 || k < 0 || i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) return -1.0f;
    const int64_t idx = ((int64_t)k * g.n[1] + j) * g.n[0] + i;
    return g.f16 ? __half2float(__ldg(reinterpret_cast<const __half*>(g.V) + idx))
                 : __ldg(reinterpret_cast<const float*>(g.V) + idx);
}

struct Dda {
    int X[3], step[3];
    float t, inv[3];
};

__device__ __forceinline__ float dda_cross(const Dda& s, const GridDev& g, const float o[3], int a) {
    if (s.step[a] == 0) return __int_as_float(0x7f800000);
    const float b = (float)(s.X[a] + (s.step[a] > 0 ? 1 : 0));
    return __fmul_rn(__fsub_rn(__fadd_rn(g.org[a], __fmul_rn(b, g.vs)), o[a]), s.inv[a]);
}

__device__ __forceinline__ bool dda_next(Dda& s, const GridDev& g, const float o[3]) {
    const float tx = dda_cross(s, g, o, 0), ty = dda_cross(s, g, o, 1), tz = dda_cross(s, g, o, 2);
    int a = 0;
    float tm = tx;
    if (ty < tm) { a = 1; tm = ty; }
    if (tz < tm) { a = 2; tm = tz; }
    s.t = tm;
    // the axis is a run-time value: update the three components by selection, so the
    // walk state stays in registers
    s.X[0] += a == 0 ? s.step[0] : 0;
    s.X[1] += a == 1 ? s.step[1] : 0;
    s.X[2] += a == 2 ? s.step[2] : 0;
    const int xa = a == 0 ? s.X[0] : (a == 1 ? s.X[1] : s.X[2]);
    const int na = a == 0 ? g.n[0] : (a == 1 ? g.n[1] : g.n[2]);
    return xa >= 0 && xa < na;
}

// walk state at parameter t0 (a point inside the grid box): the voxel containing
// o + t0 d (clamped into the grid), the step direction and 1/d of each axis
__device__ __forceinline__ void dda_init(Dda& s, const GridDev& g, const float o[3], const float d[3], float t0) {
    const float kInf = __int_as_float(0x7f800000);
    s.t = t0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        s.step[a] = d[a] > 0.0f ? 1 : (d[a] < 0.0f ? -1 : 0);
        s.inv[a] = d[a] != 0.0f ? __fdiv_rn(1.0f, d[a]) : kInf;
        const float pa = __fadd_rn(o[a], __fmul_rn(t0, d[a]));
        const float gg = floorf(__fdiv_rn(__fsub_rn(pa, g.org[a]), g.vs));
        s.X[a] = gg >= 0.0f ? (gg > (float)(g.n[a] - 1) ? g.n[a] - 1 : (int)gg) : 0;
    }
}

__device__ __forceinline__ void point_at(const float o[3], const float d[3], float t, float p[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) p[a] = __fadd_rn(o[a], __fmul_rn(t, d[a]));
}

// clip a ray to the grid box ("RenderingCube") within [t_near, t_far]: [t0, t_end]
__device__ __forceinline__ bool clip_box(const GridDev& g, const float o[3], const float d[3], float t_near, float t_far,
                                         float& t0, float& t_end) {
    const float kInf = __int_as_float(0x7f800000);
    float tmin = -kInf, tmax = kInf;
    bool hit = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = g.org[a], hi = __fadd_rn(g.org[a], __fmul_rn((float)g.n[a], g.vs));
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

}  // namespace
}  // namespace tsdfs
