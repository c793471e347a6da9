/* CPU oracle for TSDF fusion and TSDF ray bounds (TSDF-Sampling, arXiv 2311.17878).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header or table
 * with the CUDA path.
 *
 * Contents (each restates the paper's definition step by step, in FP64, and a
 * second time in the fp32-exact mode described in orc_impl.h):
 *   orc_integrate_projective_{f64,f32}  Eq. 3 + Alg. 2, per-voxel projective form
 *   orc_integrate_raycast_f64           Alg. 2 as printed: march each training ray
 *   orc_integrate_raycast_batched_{f64,f32}  the same, each view's rays applied together
 *   orc_ray_bounds_{f64,f32}            Alg. 1 (near / far phases) + Sec. 3.4 count
 *   orc_dda_sequence_{f64,f32}          the voxel walk of Alg. 1 ("NextVoxel")
 *   orc_inside_mask_{f64,f32}           Alg. 1's neighbourhood test for every voxel
 *
 * Readings of the paper that these functions take (w = 1 weights, normalised
 * storage, nearest pixel, ranges, AABB start, tie order, unseen neighbours)
 * are listed in the design notes of the repository.
 */
#include <math.h>
#include <stdlib.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

/* IEEE binary16 <-> binary32, round to nearest even (for fp16 grid storage). */
static uint16_t orc_f32_to_f16(float f)
{
    uint32_t x;
    memcpy(&x, &f, 4);
    uint32_t sign = (x >> 16) & 0x8000u;
    uint32_t ax = x & 0x7FFFFFFFu;
    if (ax >= 0x7F800000u) return (uint16_t)(sign | (ax > 0x7F800000u ? 0x7E00u : 0x7C00u));
    if (ax >= 0x477FF000u) return (uint16_t)(sign | 0x7C00u);  /* rounds to >= 65520: inf */
    if (ax < 0x38800000u) {                                    /* below 2^-14: subnormal half */
        if (ax < 0x33000000u) return (uint16_t)sign;            /* < 2^-25 rounds to 0 */
        uint32_t e = ax >> 23;
        uint32_t m = (ax & 0x7FFFFFu) | 0x800000u;
        uint32_t shift = 126u - e;                              /* 14 - (e - 127) + 23 - 10 */
        uint32_t q = m >> shift;
        uint32_t rem = m & ((1u << shift) - 1u);
        uint32_t half = 1u << (shift - 1u);
        if (rem > half || (rem == half && (q & 1u))) q += 1u;
        return (uint16_t)(sign | q);
    }
    uint32_t e = (ax >> 23) - 112u;                             /* rebias 127 -> 15 */
    uint32_t m = ax & 0x7FFFFFu;
    uint32_t q = (e << 10) | (m >> 13);
    uint32_t rem = m & 0x1FFFu;
    if (rem > 0x1000u || (rem == 0x1000u && (q & 1u))) q += 1u;
    return (uint16_t)(sign | q);
}

static float orc_f16_to_f32(uint16_t h)
{
    uint32_t sign = ((uint32_t)h & 0x8000u) << 16;
    uint32_t e = ((uint32_t)h >> 10) & 0x1Fu;
    uint32_t m = (uint32_t)h & 0x3FFu;
    uint32_t x;
    if (e == 0) {
        if (m == 0) x = sign;
        else {
            int sh = 0;
            while (!(m & 0x400u)) { m <<= 1; ++sh; }
            m &= 0x3FFu;
            x = sign | ((uint32_t)(113 - sh) << 23) | (m << 13);
        }
    } else if (e == 31) x = sign | 0x7F800000u | (m << 13);
    else x = sign | ((e + 112u) << 23) | (m << 13);
    float f;
    memcpy(&f, &x, 4);
    return f;
}

uint16_t orc_half_from_float(float f) { return orc_f32_to_f16(f); }
float orc_float_from_half(uint16_t h) { return orc_f16_to_f32(h); }

#define R double
#define SFX(name) name##_f64
#define R_SQRT sqrt
#define R_FLOOR floor
#define R_CEIL ceil
#include "orc_impl.h"
#undef R
#undef SFX
#undef R_SQRT
#undef R_FLOOR
#undef R_CEIL

#define R float
#define SFX(name) name##_f32
#define R_SQRT sqrtf
#define R_FLOOR floorf
#define R_CEIL ceilf
#include "orc_impl.h"
#undef R
#undef SFX
#undef R_SQRT
#undef R_FLOOR
#undef R_CEIL

/* ---- Alg. 2 as printed: march every training ray through the grid ---------
 * For ray (o_i, v_ij) with depth D_ij: p* = o + D v; starting at t = 0
 * (clipped to the grid box), visit voxels X with the DDA; s_X = clamp(v.(p* -
 * c_X), -D_T, D_T); if s_X > -D_T the running weighted mean is updated (w = 1)
 * and the march continues, else the ray stops.  FP64, V normalised by D_T.    */
void orc_integrate_raycast_f64(int nx, int ny, int nz, const double* origin, double vs, double trunc,
                               const float* depth, int nv, int H, int Wd, const float* K, const float* c2w,
                               double* V, uint8_t* Wt)
{
    const int n[3] = {nx, ny, nz};
    double org[3] = {origin[0], origin[1], origin[2]}, lo[3], hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = org[a]; hi[a] = org[a] + n[a] * vs; }
    for (int view = 0; view < nv; ++view) {
        const float* P = c2w + 12 * view;
        double fx = K[4 * view], fy = K[4 * view + 1], cx = K[4 * view + 2], cy = K[4 * view + 3];
        double o[3] = {P[3], P[7], P[11]};
        for (int py = 0; py < H; ++py)
            for (int px = 0; px < Wd; ++px) {
                double dc[3] = {(px + 0.5 - cx) / fx, (py + 0.5 - cy) / fy, 1.0};
                double d[3];
                for (int a = 0; a < 3; ++a) d[a] = P[4 * a] * dc[0] + P[4 * a + 1] * dc[1] + P[4 * a + 2] * dc[2];
                double nn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                for (int a = 0; a < 3; ++a) d[a] /= nn;
                double D = depth[((size_t)view * H + py) * Wd + px];
                double t0, t_end;
                if (!clip_aabb_f64(o, d, lo, hi, 0.0, INFINITY, &t0, &t_end)) continue;
                dda_t_f64 s;
                dda_init_f64(&s, o, d, org, vs, n, t0);
                int ok = 1;
                while (ok && s.t < t_end) {
                    double c[3];
                    for (int a = 0; a < 3; ++a) c[a] = org[a] + (s.X[a] + 0.5) * vs;
                    double sx;
                    if (isinf(D)) sx = trunc;
                    else {
                        double dot = 0.0;
                        for (int a = 0; a < 3; ++a) dot += d[a] * (o[a] + D * d[a] - c[a]);
                        sx = dot > trunc ? trunc : (dot < -trunc ? -trunc : dot);
                    }
                    if (!(sx > -trunc)) break;
                    size_t idx = ((size_t)s.X[2] * ny + s.X[1]) * nx + s.X[0];
                    double Wf = Wt[idx];
                    V[idx] = (Wf * V[idx] + sx / trunc) / (Wf + 1.0);
                    if (Wt[idx] < 255) Wt[idx] += 1;
                    ok = dda_next_f64(&s);
                }
            }
    }
}
