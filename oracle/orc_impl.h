/* Oracle body, instantiated twice by tsdf_oracle.c:
 *   R = double  -> the reference definition in FP64;
 *   R = float   -> the "fp32-exact" mode: IEEE binary32, round-to-nearest, no
 *                  contraction (compiled with -ffp-contract=off), every
 *                  operation in the order written here, so integer decisions
 *                  (pixel, voxel, step and sample counts) are reproducible.
 * TEST INFRASTRUCTURE ONLY: nothing in the product path may call this.
 * Requires: R, SFX(name) (suffixes names), R_SQRT, R_FLOOR, R_CEIL.
 */

/* ---- grid value access --------------------------------------------------- */
/* V is the normalised TSDF (s / D_T in [-1, 1], -1 = unseen), x fastest.      */
static R SFX(grid_at)(const void* V, int f16, int nx, int ny, int nz, int i, int j, int k)
{
    if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) return (R)-1; /* unseen */
    size_t idx = ((size_t)k * ny + j) * nx + i;
    if (f16) return (R)orc_f16_to_f32(((const uint16_t*)V)[idx]);
    return (R)((const float*)V)[idx];
}

/* ---- Eq. 3 + Alg. 2 (projective form): one voxel, all views in order --------
 * For voxel centre c and each view: x_cam = R^T (c - o); skip if z <= 0;
 * u = fx*(x/z)+cx, v = fy*(y/z)+cy; skip if outside the image; pixel
 * (floor u, floor v); D = range stored there; v_px = unit ray through that
 * pixel centre; s = clamp(D - v_px.(c - o), -D_T, D_T); if s > -D_T:
 * V <- (W V + s/D_T)/(W + 1), W <- min(W + 1, 255) (weight function w = 1).  */
static void SFX(fuse_voxel)(const R c[3], R trunc, const float* depth, int nv, int H, int Wd,
                            const float* K, const float* c2w, R* Vio, int* Wio)
{
    R Vv = *Vio;
    int Wv = *Wio;
    for (int view = 0; view < nv; ++view) {
        const float* P = c2w + 12 * view;
        R dx = c[0] - (R)P[3], dy = c[1] - (R)P[7], dz = c[2] - (R)P[11];
        R xc = ((R)P[0] * dx + (R)P[4] * dy) + (R)P[8] * dz;
        R yc = ((R)P[1] * dx + (R)P[5] * dy) + (R)P[9] * dz;
        R zc = ((R)P[2] * dx + (R)P[6] * dy) + (R)P[10] * dz;
        if (!(zc > (R)0)) continue;
        R fx = (R)K[4 * view + 0], fy = (R)K[4 * view + 1], cx = (R)K[4 * view + 2], cy = (R)K[4 * view + 3];
        R u = fx * (xc / zc) + cx;
        R v = fy * (yc / zc) + cy;
        if (!(u >= (R)0 && u < (R)Wd && v >= (R)0 && v < (R)H)) continue;
        int px = (int)R_FLOOR(u), py = (int)R_FLOOR(v);
        if (px >= Wd) px = Wd - 1;   /* cannot happen for u < W; kept for safety */
        if (py >= H) py = H - 1;
        R D = (R)depth[((size_t)view * H + py) * Wd + px];
        R a = ((R)px + (R)0.5 - cx) / fx;
        R b = ((R)py + (R)0.5 - cy) / fy;
        R nrm = R_SQRT((a * a + b * b) + (R)1);
        R proj = ((a * xc + b * yc) + zc) / nrm;
        R s = D - proj;
        if (s > trunc) s = trunc;
        if (s < -trunc) s = -trunc;
        if (s > -trunc) {
            R sn = s / trunc;
            R Wf = (R)Wv;
            Vv = (Wf * Vv + sn) / (Wf + (R)1);
            if (Wv < 255) Wv += 1;
        }
    }
    *Vio = Vv;
    *Wio = Wv;
}

/* Fuse the listed voxels (vox = NULL: all, x fastest).  V/W are in/out and are
 * indexed by position in the list.  V is R* (f16 = 0) or uint16 half bits; a
 * half value is widened on entry, carried in R across all views of the call and
 * rounded to half (nearest even) once on exit.                                */
void SFX(orc_integrate_projective)(int nx, int ny, int nz, const double* origin, double vs_d, double trunc_d,
                                   const float* depth, int nv, int H, int Wd, const float* K, const float* c2w,
                                   const int64_t* vox, int64_t n_vox, void* V, uint8_t* Wt, int f16)
{
    R vs = (R)vs_d, trunc = (R)trunc_d, org[3] = {(R)origin[0], (R)origin[1], (R)origin[2]};
    int64_t n = vox ? n_vox : (int64_t)nx * ny * nz;
    for (int64_t q = 0; q < n; ++q) {
        int64_t lin = vox ? vox[q] : q;
        int i = (int)(lin % nx), j = (int)((lin / nx) % ny), k = (int)(lin / ((int64_t)nx * ny));
        R c[3] = {org[0] + ((R)i + (R)0.5) * vs, org[1] + ((R)j + (R)0.5) * vs, org[2] + ((R)k + (R)0.5) * vs};
        R Vv = f16 ? (R)orc_f16_to_f32(((uint16_t*)V)[q]) : ((R*)V)[q];
        int Wv = Wt[q];
        SFX(fuse_voxel)(c, trunc, depth, nv, H, Wd, K, c2w, &Vv, &Wv);
        if (f16) ((uint16_t*)V)[q] = orc_f32_to_f16((float)Vv);
        else ((R*)V)[q] = Vv;
        Wt[q] = (uint8_t)Wv;
    }
}

/* ---- ray / AABB clip (the march domain, "RenderingCube") ------------------- */
static int SFX(clip_aabb)(const R o[3], const R d[3], const R lo[3], const R hi[3], R t_near, R t_far,
                          R* t0, R* t_end)
{
    R tmin = -(R)INFINITY, tmax = (R)INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == (R)0) {
            if (o[a] < lo[a] || o[a] > hi[a]) return 0;
            continue;
        }
        R inv = (R)1 / d[a];
        R t1 = (lo[a] - o[a]) * inv, t2 = (hi[a] - o[a]) * inv;
        R tl = t1 < t2 ? t1 : t2, th = t1 < t2 ? t2 : t1;
        if (tl > tmin) tmin = tl;
        if (th < tmax) tmax = th;
    }
    *t0 = t_near > tmin ? t_near : tmin;
    *t_end = t_far < tmax ? t_far : tmax;
    return *t0 < *t_end;
}

/* ---- voxel DDA ("Voxel" / "NextVoxel" of Alg. 1) ---------------------------
 * Crossing parameters are recomputed from the integer boundary each step:
 * t_a = (origin_a + (X_a + [step_a > 0]) * vs - o_a) * (1 / d_a).
 * NextVoxel takes the axis with the smallest t_a, ties to the lowest axis.    */
typedef struct {
    int X[3], step[3], n[3];
    R t, inv[3], org[3], o[3], vs;
} SFX(dda_t);

static R SFX(dda_cross)(const SFX(dda_t)* s, int a)
{
    if (s->step[a] == 0) return (R)INFINITY;
    R b = (R)(s->X[a] + (s->step[a] > 0 ? 1 : 0));
    return ((s->org[a] + b * s->vs) - s->o[a]) * s->inv[a];
}

static void SFX(dda_init)(SFX(dda_t)* s, const R o[3], const R d[3], const R org[3], R vs, const int n[3], R t0)
{
    s->t = t0;
    s->vs = vs;
    for (int a = 0; a < 3; ++a) {
        s->o[a] = o[a];
        s->org[a] = org[a];
        s->n[a] = n[a];
        s->step[a] = d[a] > (R)0 ? 1 : (d[a] < (R)0 ? -1 : 0);
        s->inv[a] = d[a] != (R)0 ? (R)1 / d[a] : (R)INFINITY;
        R p = o[a] + t0 * d[a];
        R g = R_FLOOR((p - org[a]) / vs);
        int X = g >= (R)0 ? (g > (R)(n[a] - 1) ? n[a] - 1 : (int)g) : 0;   /* NaN -> 0 */
        s->X[a] = X;
    }
}

/* advance; returns 0 when the new voxel is outside the grid */
static int SFX(dda_next)(SFX(dda_t)* s)
{
    R tx = SFX(dda_cross)(s, 0), ty = SFX(dda_cross)(s, 1), tz = SFX(dda_cross)(s, 2);
    int a = 0;
    R tm = tx;
    if (ty < tm) { a = 1; tm = ty; }
    if (tz < tm) { a = 2; tm = tz; }
    s->t = tm;
    s->X[a] += s->step[a];
    return s->X[a] >= 0 && s->X[a] < s->n[a];
}

/* trilinear TSDF on the voxel-centre lattice, clamp-to-edge, weights ignored */
static R SFX(trilinear)(const void* V, int f16, const int n[3], const R org[3], R vs, const R p[3])
{
    int i0[3];
    R fr[3];
    for (int a = 0; a < 3; ++a) {
        R g = (p[a] - org[a]) / vs - (R)0.5;
        R fl = R_FLOOR(g);
        fr[a] = g - fl;
        if (!(fl >= (R)-1)) { fl = (R)-1; fr[a] = (R)1; }   /* also NaN */
        if (fl > (R)n[a]) { fl = (R)n[a]; fr[a] = (R)0; }
        i0[a] = (int)fl;
    }
    R c[2][2][2];
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                int ii = i0[0] + dx, jj = i0[1] + dy, kk = i0[2] + dz;
                ii = ii < 0 ? 0 : (ii >= n[0] ? n[0] - 1 : ii);
                jj = jj < 0 ? 0 : (jj >= n[1] ? n[1] - 1 : jj);
                kk = kk < 0 ? 0 : (kk >= n[2] ? n[2] - 1 : kk);
                c[dz][dy][dx] = SFX(grid_at)(V, f16, n[0], n[1], n[2], ii, jj, kk);
            }
    R x00 = c[0][0][0] + fr[0] * (c[0][0][1] - c[0][0][0]);
    R x01 = c[0][1][0] + fr[0] * (c[0][1][1] - c[0][1][0]);
    R x10 = c[1][0][0] + fr[0] * (c[1][0][1] - c[1][0][0]);
    R x11 = c[1][1][0] + fr[0] * (c[1][1][1] - c[1][1][0]);
    R y0 = x00 + fr[1] * (x01 - x00);
    R y1 = x10 + fr[1] * (x11 - x10);
    return y0 + fr[2] * (y1 - y0);
}

/* "ForAll(NeighborVoxels, V < 0)" of Alg. 1, radius r around X; out-of-grid
 * neighbours read as unseen (-1).                                             */
static int SFX(all_negative)(const void* V, int f16, const int n[3], const int X[3], int r)
{
    for (int dz = -r; dz <= r; ++dz)
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx)
                if (!(SFX(grid_at)(V, f16, n[0], n[1], n[2], X[0] + dx, X[1] + dy, X[2] + dz) < (R)0)) return 0;
    return 1;
}

/* ---- Alg. 1: sample bounds of one ray, then the adaptive count (Sec. 3.4) ---
 * status: 0 MISS (no overlap with the grid box / [t_near, t_far]), 1 BOUNDED,
 * 2 FALLBACK (no voxel satisfies V <= D_s: the whole [t0, t_end] with
 * n_fallback samples).  steps = number of voxels tested (near + far).        */
void SFX(orc_ray_bounds)(int nx, int ny, int nz, const double* origin, double vs_d, double trunc_d,
                         const void* V, int f16, const float* ray_o, const float* ray_d, int64_t n_rays,
                         double d_s, double t_near, double t_far, double step, int nb_radius, int m_confirm,
                         int n_max, int n_fallback,
                         R* t_n_out, R* t_f_out, int32_t* n_out, R* t_zero_out, uint8_t* status_out,
                         int32_t* steps_out)
{
    const int n[3] = {nx, ny, nz};
    R vs = (R)vs_d, trunc = (R)trunc_d;
    R org[3] = {(R)origin[0], (R)origin[1], (R)origin[2]};
    R lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = org[a];
        hi[a] = org[a] + (R)n[a] * vs;
    }
    R ds_norm = (R)d_s / trunc;
    R stepR = (R)step;
    for (int64_t r = 0; r < n_rays; ++r) {
        R o[3] = {(R)ray_o[3 * r], (R)ray_o[3 * r + 1], (R)ray_o[3 * r + 2]};
        R d[3] = {(R)ray_d[3 * r], (R)ray_d[3 * r + 1], (R)ray_d[3 * r + 2]};
        R t0, t_end;
        int steps = 0;
        if (!SFX(clip_aabb)(o, d, lo, hi, (R)t_near, (R)t_far, &t0, &t_end)) {
            t_n_out[r] = 0; t_f_out[r] = 0; n_out[r] = 0; t_zero_out[r] = (R)NAN; status_out[r] = 0;
            if (steps_out) steps_out[r] = 0;
            continue;
        }
        SFX(dda_t) s;
        SFX(dda_init)(&s, o, d, org, vs, n, t0);
        /* near phase: first voxel whose centre value is <= D_s */
        int found = 0, inside_grid = 1;
        R t_before = t0;   /* entry of the voxel before the current one (t0 for the first) */
        while (inside_grid && s.t < t_end) {
            ++steps;
            if (SFX(grid_at)(V, f16, nx, ny, nz, s.X[0], s.X[1], s.X[2]) <= ds_norm) { found = 1; break; }
            t_before = s.t;
            inside_grid = SFX(dda_next)(&s);
        }
        if (!found) {
            t_n_out[r] = t0; t_f_out[r] = t_end; n_out[r] = n_fallback; t_zero_out[r] = (R)NAN; status_out[r] = 2;
            if (steps_out) steps_out[r] = steps;
            continue;
        }
        R tn = s.t, tf = t_end;
        /* zero-crossing search: trilinear TSDF at the crossing points from the
         * entry of the voxel before the near voxel up to t_f; the first +/- sign
         * change gives the secant root t_zero (NaN if there is none)        */
        R tz = (R)NAN, t_prev = t_before, v_prev;
        {
            R p[3] = {o[0] + t_before * d[0], o[1] + t_before * d[1], o[2] + t_before * d[2]};
            v_prev = SFX(trilinear)(V, f16, n, org, vs, p);
            R pn[3] = {o[0] + tn * d[0], o[1] + tn * d[1], o[2] + tn * d[2]};
            R vn = SFX(trilinear)(V, f16, n, org, vs, pn);
            if (tn > t_before && v_prev > (R)0 && vn <= (R)0) tz = t_prev + (tn - t_prev) * (v_prev / (v_prev - vn));
            v_prev = vn;
            t_prev = tn;
        }
        /* far phase: the first test is on the same voxel */
        int m = 0;
        while (inside_grid && s.t < t_end) {
            ++steps;
            int inside = SFX(all_negative)(V, f16, n, s.X, nb_radius);
            m = inside ? m + 1 : 0;
            inside_grid = SFX(dda_next)(&s);
            R tc = s.t < t_end ? s.t : t_end;
            if (tz != tz) {
                R p[3] = {o[0] + tc * d[0], o[1] + tc * d[1], o[2] + tc * d[2]};
                R vc = SFX(trilinear)(V, f16, n, org, vs, p);
                if (v_prev > (R)0 && vc <= (R)0) tz = t_prev + (tc - t_prev) * (v_prev / (v_prev - vc));
                v_prev = vc;
                t_prev = tc;
            }
            if (m == m_confirm) { tf = tc; break; }
        }
        R L = tf - tn;
        R q = L / stepR;
        int cnt;
        if (!(q > (R)1)) cnt = 1;
        else if (q >= (R)n_max) cnt = n_max;
        else cnt = (int)R_CEIL(q);
        if (cnt > n_max) cnt = n_max;
        t_n_out[r] = tn; t_f_out[r] = tf; n_out[r] = cnt; t_zero_out[r] = tz; status_out[r] = 1;
        if (steps_out) steps_out[r] = steps;
    }
}

/* Voxel sequence the DDA visits from t0 until it leaves the grid or passes
 * t_end (for the brute-force intersection pin).  Returns the count written.  */
int64_t SFX(orc_dda_sequence)(int nx, int ny, int nz, const double* origin, double vs_d, const float* o_in,
                              const float* d_in, double t_near, double t_far, int32_t* xyz_out, R* t_out,
                              int64_t cap)
{
    const int n[3] = {nx, ny, nz};
    R vs = (R)vs_d, org[3] = {(R)origin[0], (R)origin[1], (R)origin[2]}, lo[3], hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = org[a]; hi[a] = org[a] + (R)n[a] * vs; }
    R o[3] = {(R)o_in[0], (R)o_in[1], (R)o_in[2]}, d[3] = {(R)d_in[0], (R)d_in[1], (R)d_in[2]};
    R t0, t_end;
    if (!SFX(clip_aabb)(o, d, lo, hi, (R)t_near, (R)t_far, &t0, &t_end)) return 0;
    SFX(dda_t) s;
    SFX(dda_init)(&s, o, d, org, vs, n, t0);
    int64_t c = 0;
    int ok = 1;
    while (ok && s.t < t_end && c < cap) {
        xyz_out[3 * c] = s.X[0]; xyz_out[3 * c + 1] = s.X[1]; xyz_out[3 * c + 2] = s.X[2];
        t_out[c] = s.t;
        ++c;
        ok = SFX(dda_next)(&s);
    }
    return c;
}

/* inside mask of the far test for every voxel, 1 byte per voxel */
void SFX(orc_inside_mask)(int nx, int ny, int nz, const void* V, int f16, int r, uint8_t* out)
{
    const int n[3] = {nx, ny, nz};
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int X[3] = {i, j, k};
                out[((size_t)k * ny + j) * nx + i] = (uint8_t)SFX(all_negative)(V, f16, n, X, r);
            }
}

/* grid-box clip of many rays: t0 = max(t_near, t_entry), t_end = min(t_far, t_exit) */
void SFX(orc_clip_rays)(int nx, int ny, int nz, const double* origin, double vs_d, const float* ray_o,
                        const float* ray_d, int64_t n_rays, double t_near, double t_far, R* t0_out, R* t_end_out,
                        uint8_t* ok_out)
{
    const int n[3] = {nx, ny, nz};
    R vs = (R)vs_d, lo[3], hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = (R)origin[a]; hi[a] = (R)origin[a] + (R)n[a] * vs; }
    for (int64_t r = 0; r < n_rays; ++r) {
        R o[3] = {(R)ray_o[3 * r], (R)ray_o[3 * r + 1], (R)ray_o[3 * r + 2]};
        R d[3] = {(R)ray_d[3 * r], (R)ray_d[3 * r + 1], (R)ray_d[3 * r + 2]};
        R t0 = 0, te = 0;
        ok_out[r] = (uint8_t)SFX(clip_aabb)(o, d, lo, hi, (R)t_near, (R)t_far, &t0, &te);
        t0_out[r] = t0;
        t_end_out[r] = te;
    }
}

/* ---- Alg. 2 as printed, the rays of one view applied together (reading R27) --
 * Views in order.  For every pixel (row-major) of a view: unit ray through the
 * pixel centre, v = normalise(R ((px + 1/2 - cx)/fx, (py + 1/2 - cy)/fy, 1)),
 * o = the camera centre, p* = o + D v (D = the stored range); clip to the grid
 * box from t = 0; voxel walk (above); at each voxel s = clamp(v . (p* - c),
 * -D_T, D_T) (D = +inf: s = D_T); stop at the first s <= -D_T, else the voxel
 * records s / D_T and one visit.  After all the view's rays, every voxel with
 * k > 0 visits: V <- (W V + sum) / (W + k), W <- min(W + k, 255).
 * FP64 mode: sum in FP64.  fp32-exact mode: s / D_T in binary32, each turned
 * into an integer number of 2^-32 units (round to nearest even) and summed
 * exactly, then the update in FP64 and one rounding to binary32 (or to half for
 * half storage, once per view).  V is R* or uint16 half bits, W uint8.       */
void SFX(orc_integrate_raycast_batched)(int nx, int ny, int nz, const double* origin, double vs_d, double trunc_d,
                                        const float* depth, int nv, int H, int Wd, const float* K, const float* c2w,
                                        void* V, uint8_t* Wt, int f16)
{
    const int n[3] = {nx, ny, nz};
    const size_t nvox = (size_t)nx * ny * nz;
    R vs = (R)vs_d, trunc = (R)trunc_d, org[3] = {(R)origin[0], (R)origin[1], (R)origin[2]}, lo[3], hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = org[a]; hi[a] = org[a] + (R)n[a] * vs; }
    const int fixed = sizeof(R) == sizeof(float);
    double* dsum = fixed ? NULL : (double*)calloc(nvox, sizeof(double));
    int64_t* qsum = fixed ? (int64_t*)calloc(nvox, sizeof(int64_t)) : NULL;
    uint32_t* cnt = (uint32_t*)calloc(nvox, sizeof(uint32_t));
    if ((!dsum && !qsum) || !cnt) { free(dsum); free(qsum); free(cnt); return; }
    for (int view = 0; view < nv; ++view) {
        const float* P = c2w + 12 * view;
        R fx = (R)K[4 * view], fy = (R)K[4 * view + 1], cx = (R)K[4 * view + 2], cy = (R)K[4 * view + 3];
        R o[3] = {(R)P[3], (R)P[7], (R)P[11]};
        for (int py = 0; py < H; ++py)
            for (int px = 0; px < Wd; ++px) {
                R a = (((R)px + (R)0.5) - cx) / fx, b = (((R)py + (R)0.5) - cy) / fy;
                R d[3];
                for (int k = 0; k < 3; ++k) d[k] = ((R)P[4 * k] * a + (R)P[4 * k + 1] * b) + (R)P[4 * k + 2];
                R nn = R_SQRT((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
                for (int k = 0; k < 3; ++k) d[k] = d[k] / nn;
                R D = (R)depth[((size_t)view * H + py) * Wd + px];
                R t0, t_end;
                if (!SFX(clip_aabb)(o, d, lo, hi, (R)0, (R)INFINITY, &t0, &t_end)) continue;
                R ps[3];
                for (int k = 0; k < 3; ++k) ps[k] = o[k] + D * d[k];
                SFX(dda_t) s;
                SFX(dda_init)(&s, o, d, org, vs, n, t0);
                int ok = 1;
                while (ok && s.t < t_end) {
                    R sx = trunc;
                    if (!isinf(D)) {
                        R e[3];
                        for (int k = 0; k < 3; ++k) e[k] = ps[k] - (org[k] + ((R)s.X[k] + (R)0.5) * vs);
                        R dot = (d[0] * e[0] + d[1] * e[1]) + d[2] * e[2];
                        sx = dot > trunc ? trunc : (dot < -trunc ? -trunc : dot);
                    }
                    if (!(sx > -trunc)) break;
                    size_t idx = ((size_t)s.X[2] * ny + s.X[1]) * nx + s.X[0];
                    R x = sx / trunc;
                    if (fixed) qsum[idx] += (int64_t)llrint((double)x * 4294967296.0);
                    else dsum[idx] += (double)x;
                    cnt[idx] += 1;
                    ok = SFX(dda_next)(&s);
                }
            }
        for (size_t q = 0; q < nvox; ++q) {
            if (!cnt[q]) continue;
            double v = f16 ? (double)orc_f16_to_f32(((uint16_t*)V)[q]) : (double)((R*)V)[q];
            double sum = fixed ? (double)qsum[q] / 4294967296.0 : dsum[q];
            double w = (double)Wt[q];
            double vn = (w * v + sum) / (w + (double)cnt[q]);
            if (f16) ((uint16_t*)V)[q] = orc_f32_to_f16((float)vn);
            else ((R*)V)[q] = (R)vn;
            uint32_t wn = (uint32_t)Wt[q] + cnt[q];
            Wt[q] = (uint8_t)(wn > 255u ? 255u : wn);
            cnt[q] = 0;
            if (fixed) qsum[q] = 0;
            else dsum[q] = 0.0;
        }
    }
    free(dsum);
    free(qsum);
    free(cnt);
}
