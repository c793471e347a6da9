/*
 * tsdfs.h -- C ABI of the GB300 (sm_103a) TSDF-Sampling library.
 *
 * TSDF-Sampling (arXiv 2311.17878) renders a neural surface field with few
 * samples per ray: a TSDF volume fused from depth maps (Sec. 3.2, Eq. 3,
 * Alg. 2) bounds each novel-view ray to an interval [t_n, t_f] around its first
 * surface (Sec. 3.3, Alg. 1); the number of samples follows the interval
 * length (Sec. 3.4); the SDF and colour networks run only there and are
 * volume rendered (Eq. 1, Eq. 2, the rendered normal of Sec. C.1).
 *
 * Conventions for every entry point:
 *  - Pointers named in a struct or argument are DEVICE pointers unless the
 *    comment says "host".  The caller owns every buffer; the library
 *    allocates and frees nothing itself (no cudaMalloc / cudaFree in it; the
 *    layer-major backward's first call on a device creates a cuBLAS handle,
 *    whose state cuBLAS allocates).  The render workspaces (render_rays,
 *    render_rays_hier, render_rays_hier_bounded) include about 10 MB for the
 *    tensor-core network kernel, which parks the first tile of each pair of
 *    64-sample tiles there (256 CTAs x 38 KB).
 *  - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL = the
 *    legacy default stream); the calls that synchronise say so (the autotuners,
 *    the layer-major backward and training forward, which read the sample
 *    total, and the FP64 harness).  Arguments are checked on the host before any
 *    launch; a check failure returns a negative TSDFS_E_* code, enqueues
 *    nothing and records a message for tsdfs_last_error().
 *  - Kernels never trap.  Conditions that only the device can see (a sample
 *    total above the workspace capacity, a march exceeding its step cap) set
 *    a bit in a device status word, read back by tsdfs_sync_status().
 *  - Arrays are row-major; xyz triples are interleaved ([n][3]); grids are
 *    x-fastest ([nz][ny][nx]).  Ray directions must be unit length (Alg. 1:
 *    "ray (unit direction vector)").
 */
#ifndef TSDFS_H
#define TSDFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* tsdfs_stream_t; /* identical to cudaStream_t */

/* ---- return codes ------------------------------------------------------- */
#define TSDFS_OK 0
#define TSDFS_E_INVALID (-1)     /* bad argument: null pointer, size, parameter  */
#define TSDFS_E_CUDA (-2)        /* a CUDA runtime call failed                   */
#define TSDFS_E_WORKSPACE (-3)   /* workspace smaller than the *_workspace_size  */
#define TSDFS_E_UNSUPPORTED (-4) /* architecture / precision combination         */
#define TSDFS_E_DEVICE (-5)      /* tsdfs_sync_status: a device-side check fired */

/* device status bits reported by tsdfs_sync_status() */
#define TSDFS_DEV_SAMPLES_OVERFLOW 1u /* offsets[n_rays] exceeded max_samples   */
#define TSDFS_DEV_MARCH_CAP 2u        /* a ray hit the voxel-step cap            */
#define TSDFS_DEV_TIMEOUT 4u          /* a bounded wait in a pipelined kernel expired */
#define TSDFS_DEV_NONFINITE 8u        /* a network parameter is NaN or infinite         */

/* ---- TSDF grid (Sec. 3.2; Sec. A.1: V initialised to -1 = unseen, W to 0) -
 * tsdf holds s / D_T in [-1, 1] (normalised truncated signed distance), as
 * float (TSDFS_F32) or IEEE half (TSDFS_F16); weight counts fused
 * observations, saturating at 255.  Voxel (i, j, k) covers
 * origin + [i, i+1) x [j, j+1) x [k, k+1) * voxel_size; its centre is at
 * origin + (i + 1/2, j + 1/2, k + 1/2) * voxel_size.                         */
#define TSDFS_F32 0
#define TSDFS_F16 1
typedef struct {
    int32_t nx, ny, nz;
    float origin[3];   /* metres, min corner of voxel (0, 0, 0)          */
    float voxel_size;  /* metres                                           */
    float trunc;       /* D_T, metres (Eq. 3)                              */
    int32_t dtype;     /* TSDFS_F32 | TSDFS_F16                            */
    void* tsdf;        /* device, nz*ny*nx values                          */
    uint8_t* weight;   /* device, nz*ny*nx                                 */
} tsdfs_grid;

/* ---- Alg. 1 / Sec. 3.4 parameters ---------------------------------------- */
typedef struct {
    float d_s;          /* D_s, surface criterion, metres (Alg. 1)                   */
    float t_near;       /* start of the original ray range                           */
    float t_far;        /* original far bound t_f of Alg. 1                           */
    float step;         /* sample spacing (metres) of the adaptive count, Sec. 3.4   */
    int32_t nb_radius;  /* neighbourhood radius: 2 -> 5x5x5 (Sec. 4.2)               */
    int32_t m_confirm;  /* M: consecutive inside voxels before t_f (Sec. 4.2: 15)    */
    int32_t n_max;      /* cap of the adaptive count                                 */
    int32_t n_fallback; /* samples over [t0, t_end] when no voxel passes V <= D_s    */
} tsdfs_bounds_params;

/* per-ray status written by tsdf_ray_bounds */
#define TSDFS_MISS 0     /* the ray does not overlap the grid box within [t_near, t_far] */
#define TSDFS_BOUNDED 1  /* [t_n, t_f] from Alg. 1                                       */
#define TSDFS_FALLBACK 2 /* no surface voxel: [t0, t_end] with n_fallback samples        */

/* ---- networks --------------------------------------------------------------
 * SDF network: input gamma(x~), x~ = (x - center) / scale, gamma the
 * positional encoding (x~, sin(2^k x~), cos(2^k x~)), k < L; hidden layers
 * softplus_beta (linear where beta z > 20); linear output [net_0, feature];
 * SDF f = scale * net_0; grad f = d net_0 / d x~.  The skip layer takes
 * concat(h, gamma) / sqrt(2).  Colour network: input (x~, direction encoding,
 * unit normal grad f / |grad f|, feature), ReLU hidden layers, sigmoid output.
 *   TSDFS_ARCH_TINY: SDF 3-64-64-64-(1+16), colour 25-64-64-3, no encodings.
 *   TSDFS_ARCH_ROOM: SDF 39-256-256-256-217, skip, 256-256-256-(1+256), L = 6;
 *                    colour (3+27+3+256)-256-256-256-256-3, direction L = 4.
 * Packed fp32 parameters (sdf_w, rgb_w): for each layer in order, W[out][in]
 * row-major, then b[out].  Opacity of a sample's section (the SDF-to-density
 * transform of the backbone in Eq. 1), by `opacity`:
 *   TSDFS_OPACITY_NEUS:   alpha = clamp((Phi(f-) - Phi(f+) + eps)/(Phi(f-) + eps),
 *                         0, 1), Phi(x) = sigmoid(inv_s x),
 *                         f-/+ = f -/+ (delta/2) min(v . grad f, 0);
 *   TSDFS_OPACITY_VOLSDF: alpha = 1 - exp(-sigma(f) delta) (Eq. 1 as printed) with
 *                         the density of VolSDF / MonoSDF, sigma(f) = a Psi(-f),
 *                         Psi the CDF of the zero-mean Laplace distribution of
 *                         scale 1/a, a = inv_s (eps unused).                    */
#define TSDFS_OPACITY_NEUS 0
#define TSDFS_OPACITY_VOLSDF 1
#define TSDFS_ARCH_TINY 0
#define TSDFS_ARCH_ROOM 1
#define TSDFS_PREC_F32 0  /* FP32 SIMT networks                                  */
#define TSDFS_PREC_BF16 1 /* BF16 tcgen05 networks, FP32 accumulate (packed required) */
#define TSDFS_PREC_F16 2  /* FP16 operands on the same tcgen05 path (packed required)  */
#define TSDFS_PREC_BF16X2 3 /* BF16 tcgen05 networks with every SDF layer's operand split
                             * into two BF16 parts, hi = bf16(x) and lo = bf16(x - hi),
                             * two MMAs per K step into the FP32 accumulator (about 16
                             * significant bits per activation); colour layers in plain
                             * BF16; packed BF16 weights required; pipelined kernel only */
typedef struct {
    int32_t arch;
    int32_t precision;
    const float* sdf_w;  /* device, packed fp32                                         */
    const float* rgb_w;  /* device, packed fp32                                         */
    const void* packed;  /* device, tsdfs_packed_size bytes from tsdfs_pack_mlp, or NULL */
    float center[3];
    float scale;
    float inv_s;         /* NeuS: s of Phi_s (64); VolSDF: a = 1/beta of the density     */
    float beta;          /* softplus beta (100)                                         */
    float alpha_eps;     /* eps of the NeuS opacity ratio (1e-5)                        */
    int32_t opacity;     /* TSDFS_OPACITY_NEUS (0) or TSDFS_OPACITY_VOLSDF (1)          */
} tsdfs_mlp;

/* ---- errors -------------------------------------------------------------- */
/* Message of the last failing call on this host thread ("" if none). */
const char* tsdfs_last_error(void);
/* Synchronise `stream`, then read and clear the device status word.  Returns
 * TSDFS_OK, TSDFS_E_DEVICE (bits in *bits_out when non-NULL) or TSDFS_E_CUDA. */
int tsdfs_sync_status(tsdfs_stream_t stream, uint32_t* bits_out);

/* ---- fusion (Sec. 3.2, Eq. 3, Alg. 2; Sec. A.1 initial values) -------------
 * tsdfs_grid_init: V = -1 (unseen), W = 0 for every voxel.
 * tsdf_integrate: per-voxel projective form of Alg. 2.  For each voxel centre
 *   c and each view in order 0..n_views-1: x_cam = R^T (c - o); skip when
 *   z <= 0; pixel (floor(fx x/z + cx), floor(fy y/z + cy)), skip when outside
 *   the image; D = depth at that pixel (range along the unit ray through the
 *   pixel centre; +inf = no surface); s = clamp(D - v_px . (c - o), -D_T, D_T);
 *   when s > -D_T: V <- (W V + s/D_T)/(W + 1), W <- min(W + 1, 255).
 *   depth: device [n_views][H][W] float; K: device [n_views][4] (fx, fy, cx,
 *   cy); c2w: device [n_views][12], row-major 3x4 [R | o], OpenCV camera axes.
 *   Runs in fp32 with round-to-nearest and no contraction, in the operation
 *   order above, so results are reproducible bit for bit.  F16 grids are
 *   widened, updated in fp32 across all views of the call and rounded once. */
int tsdfs_grid_init(const tsdfs_grid* grid, tsdfs_stream_t stream);
int tsdf_integrate(const tsdfs_grid* grid, const float* depth, int32_t n_views, int32_t height, int32_t width,
                   const float* K, const float* c2w, tsdfs_stream_t stream);

/* tsdf_integrate_raycast: Alg. 2 as printed, marching every training ray.
 *   Views in order; for each pixel of a view: v = the unit ray through the
 *   pixel centre, normalise(R ((px + 1/2 - cx)/fx, (py + 1/2 - cy)/fy, 1)),
 *   o = the camera centre, p* = o + D v (D = the stored range); the ray is
 *   clipped to the grid box from t = 0 and walked voxel by voxel (the walk of
 *   tsdf_ray_bounds); at each voxel s = clamp(v . (p* - c), -D_T, D_T)
 *   (D = +inf: s = D_T); the walk stops at the first s <= -D_T, else the voxel
 *   records s / D_T and one visit.  The rays of one view are applied together:
 *   every voxel with k > 0 visits gets V <- (W V + sum) / (W + k),
 *   W <- min(W + k, 255) (for w = 1 and no saturation this equals the one-ray-
 *   at-a-time running mean).  Each s / D_T is summed as an integer number of
 *   2^-32 units (round to nearest even), exactly and in any order, and the
 *   update is done in FP64 and rounded once (to half, per view, for half
 *   storage): results are reproducible bit for bit.  Rays and walk in fp32
 *   with round-to-nearest and no contraction.  At most 2^21 pixels per view.
 *   Arguments as tsdf_integrate; workspace >= tsdfs_raycast_workspace_size
 *   (12 bytes per voxel).                                                   */
size_t tsdfs_raycast_workspace_size(const tsdfs_grid* grid);
int tsdf_integrate_raycast(const tsdfs_grid* grid, const float* depth, int32_t n_views, int32_t height,
                           int32_t width, const float* K, const float* c2w, void* workspace, size_t ws_bytes,
                           tsdfs_stream_t stream);

/* ---- far-phase neighbourhood test, precomputed (Alg. 1) ---------------------
 * bit (k*ny + j)*nx + i of mask_bits (uint32 words, little bit order) is 1 iff
 * every voxel within Chebyshev radius nb_radius of (i, j, k) has V < 0 (out of
 * grid = unseen = -1).  mask_bits: device, tsdfs_inside_mask_words() words.
 * Optional input of tsdf_ray_bounds; results are identical with or without. */
int64_t tsdfs_inside_mask_words(const tsdfs_grid* grid);
int tsdfs_inside_mask(const tsdfs_grid* grid, int32_t nb_radius, uint32_t* mask_bits, tsdfs_stream_t stream);

/* ---- ray bounds (Alg. 1) and adaptive count (Sec. 3.4) ----------------------
 * Per ray: [t0, t_end] = [t_near, t_far] clipped to the grid box (MISS if
 * empty).  Voxel walk from t0 (crossing parameters recomputed from integer
 * boundaries, ties x < y < z).  Near phase: first voxel X with
 * V(centre X) <= d_s / D_T gives t_n = its entry parameter; none: FALLBACK.
 * Far phase from the same X: m counts consecutive voxels whose neighbourhood
 * is all negative; when m reaches m_confirm after a step, t_f = the entry of
 * the next voxel (capped at t_end); else t_f = t_end.  Count n = clamp(ceil(
 * (t_f - t_n)/step), 1, n_max); FALLBACK: t_n = t0, t_f = t_end, n =
 * n_fallback; MISS: n = 0, t_n = t_f = 0.  t_zero: first +/- sign change of
 * the trilinear TSDF at the crossing points from the entry of the voxel before
 * the near voxel to t_f, secant root; NaN if none or not BOUNDED.
 * offsets[0..n_rays] = exclusive prefix sum of n (offsets[n_rays] = total).
 * inside_mask: NULL or the output of tsdfs_inside_mask for p->nb_radius.
 * t_zero may be NULL.  workspace: device, >= tsdfs_bounds_workspace_size.
 * Integer results and t_n / t_f equal the fp32-exact reference bit for bit. */
size_t tsdfs_bounds_workspace_size(int64_t n_rays);
int tsdf_ray_bounds(const tsdfs_grid* grid, const uint32_t* inside_mask, const float* ray_o, const float* ray_d,
                    int64_t n_rays, const tsdfs_bounds_params* p, float* t_n, float* t_f, int32_t* n_samples,
                    int32_t* offsets, float* t_zero, uint8_t* status, void* workspace, size_t ws_bytes,
                    tsdfs_stream_t stream);

/* ---- ray bounds for callers that cannot allocate (no counterpart in the paper)
 * Same computation, arguments and results as tsdf_ray_bounds, without the
 * workspace: for callers that cannot allocate device memory themselves (a
 * host application that only hands over buffers it registered up front, a
 * real-time loop that must not allocate once running, code inside a framework
 * whose allocator it cannot reach).  The offsets scan's scratch is a
 * file-scope device array of the library, present on every device that loads
 * it until the process exits, sized for tsdf_ray_bounds_noalloc_max_rays()
 * (2^24) rays per call; larger n_rays is rejected with TSDFS_E_INVALID.  The
 * first call on a device looks up that array's address (cudaGetSymbolAddress)
 * and should therefore come before any stream capture.  The call allocates
 * and frees nothing.  All calls share the array: calls that overlap on the GPU
 * (unordered streams) race on it and must be serialised by the caller.       */
int64_t tsdf_ray_bounds_noalloc_max_rays(void);
int tsdf_ray_bounds_noalloc(const tsdfs_grid* grid, const uint32_t* inside_mask, const float* ray_o,
                            const float* ray_d, int64_t n_rays, const tsdfs_bounds_params* p, float* t_n, float* t_f,
                            int32_t* n_samples, int32_t* offsets, float* t_zero, uint8_t* status,
                            tsdfs_stream_t stream);

/* ---- render (Sec. 3.4 placement; Eq. 1, Eq. 2; rendered normal Sec. C.1) ----
 * Ray r has offsets[r+1] - offsets[r] samples at the midpoints
 * t_i = t_n + (i + 1/2)(t_f - t_n)/n of [t_n, t_f] (FALLBACK rays carry
 * [t0, t_end] and n_fallback from tsdf_ray_bounds).  Per sample: SDF network
 * value f, gradient, feature; colour network; NeuS opacity with section width
 * (t_f - t_n)/n.  Compositing: log T_0 = 0, log T_{i+1} = log T_i +
 * log1p(-min(alpha_i, 1 - 2^-24)), w_i = exp(log T_i) alpha_i; rgb = sum w c
 * (black background); wsum = sum w; depth = sum w t / wsum and normal =
 * sum w n / wsum (both 0 when wsum < 1e-8).  Rays with zero samples give 0.
 * eik (nullable): per-ray sum over samples of (|grad f| - 1)^2, written only
 * for BOUNDED rays (0 otherwise).  normal may be NULL.
 * max_samples bounds offsets[n_rays]; workspace >= tsdfs_render_workspace_size.
 * precision TSDFS_PREC_BF16 / TSDFS_PREC_F16 / TSDFS_PREC_BF16X2 needs
 * mlp->packed from tsdfs_pack_mlp (packed for that precision).              */
size_t tsdfs_render_workspace_size(const tsdfs_mlp* mlp, int64_t n_rays, int64_t max_samples);
int render_rays(const tsdfs_mlp* mlp, const float* ray_o, const float* ray_d, const float* t_n, const float* t_f,
                const int32_t* offsets, const uint8_t* status, int64_t n_rays, int64_t max_samples, float* rgb,
                float* depth, float* wsum, float* normal, float* eik, void* workspace, size_t ws_bytes,
                tsdfs_stream_t stream);

/* ---- recovery of rays the bounds missed (Sec. 4.5, threshold tau of Tab. 5) ----
 * A second pass for rays whose accumulated weight stays low: every BOUNDED ray
 * r with wsum[r] < tau (wsum from a first render_rays) gets status2 =
 * TSDFS_FALLBACK, [t_n2, t_f2] = [t0, t_end] (its grid-box clip of
 * [t_near, t_far], fp32 as in tsdf_ray_bounds) and n2 = p->n_fallback; every
 * other ray (MISS, FALLBACK, or wsum >= tau) gets n2 = 0, status2 = TSDFS_MISS,
 * t_n2 = t_f2 = 0.  offsets2 is the exclusive scan of n2 (n_rays + 1 entries).
 * Render the second pass with render_rays(t_n2, t_f2, offsets2, status2) into
 * separate outputs, then tsdf_recovery_merge.  All arrays are device memory,
 * caller-owned, ray-major as in tsdf_ray_bounds; p->d_s, step, n_max,
 * nb_radius and m_confirm are not used.  ws >= tsdfs_bounds_workspace_size.
 * Asynchronous on stream; argument errors return negative codes.            */
int tsdf_recovery_bounds(const tsdfs_grid* grid, const float* ray_o, const float* ray_d, int64_t n_rays,
                         const tsdfs_bounds_params* p, float tau, const float* wsum, const uint8_t* status,
                         float* t_n2, float* t_f2, int32_t* n2, int32_t* offsets2, uint8_t* status2, void* ws,
                         size_t ws_bytes, tsdfs_stream_t stream);
/* Copy the second render's rgb[3], depth, wsum (and normal[3] when both normal
 * pointers are non-NULL; both or neither) over the first render's outputs for
 * the rays with status2 == TSDFS_FALLBACK.  Device pointers, in place.       */
int tsdf_recovery_merge(int64_t n_rays, const uint8_t* status2, const float* rgb2, const float* depth2,
                        const float* wsum2, const float* normal2, float* rgb, float* depth, float* wsum,
                        float* normal, tsdfs_stream_t stream);

/* ---- hierarchical comparator (n_c coarse + n_f inverse-CDF fine; 64 + 32 is
 * the "HS" sampler of Tab. 2) ------------------------------------------------
 * Per ray over [t0, t_end] (t_near/t_far clipped to the grid box of `grid`;
 * only its geometry fields are read): n_c midpoints, SDF values only; section
 * weights from the values (NeuS up-sampling opacity: slope min(own,
 * previous), clipped to [-1e3, 0]); n_f inverse-CDF samples at
 * u = (k+1/2)/n_f over pdf ~ w + 1e-5; all n_c + n_f sorted samples evaluated
 * fully and composited with section boundaries halfway between neighbours.
 * Outputs as render_rays.  2 <= n_coarse <= 64, 1 <= n_fine <= 32, else
 * TSDFS_E_INVALID.  workspace >= tsdfs_hier_workspace_size (sized for 64 + 32,
 * so it serves every count).  render_rays_hier96 is n_coarse = 64,
 * n_fine = 32.                                                              */
size_t tsdfs_hier_workspace_size(const tsdfs_mlp* mlp, int64_t n_rays);
int render_rays_hier(const tsdfs_mlp* mlp, const tsdfs_grid* grid, const float* ray_o, const float* ray_d,
                     int64_t n_rays, int n_coarse, int n_fine, float t_near, float t_far, float* rgb, float* depth,
                     float* wsum, float* normal, void* workspace, size_t ws_bytes, tsdfs_stream_t stream);
int render_rays_hier96(const tsdfs_mlp* mlp, const tsdfs_grid* grid, const float* ray_o, const float* ray_d,
                       int64_t n_rays, float t_near, float t_far, float* rgb, float* depth, float* wsum,
                       float* normal, void* workspace, size_t ws_bytes, tsdfs_stream_t stream);

/* ---- launch shape of the march and its autotuner --------------------------
 * tsdf_ray_bounds and tsdf_recovery_bounds launch a grid-stride march of
 * `block` threads per block and at most `blocks_per_sm` blocks per SM (default
 * 128 and 64).  Outputs do not depend on the shape (rays are independent);
 * speed does.  tsdfs_autotune_bounds times every candidate (block in {64, 128,
 * 256} x blocks_per_sm in {4, 8, 16, 32, 64}) with CUDA events on `stream`,
 * `reps` launches each of tsdf_ray_bounds on the caller's rays and buffers
 * (arguments as tsdf_ray_bounds; the outputs hold the last run's results), and
 * keeps the fastest as this device's shape; best_ms (host, or NULL) receives
 * its time per launch.  It synchronises the stream: call it at set-up, not
 * inside a captured step.  tsdfs_set_bounds_launch_shape sets a shape
 * directly (0, 0 = the default; block a multiple of 32 in [32, 256],
 * blocks_per_sm in [1, 1024]); tsdfs_bounds_launch_shape reads it.  The shape
 * is per device and process-wide.                                            */
int tsdfs_autotune_bounds(const tsdfs_grid* grid, const uint32_t* inside_mask, const float* ray_o, const float* ray_d,
                          int64_t n_rays, const tsdfs_bounds_params* params, float* t_n, float* t_f,
                          int32_t* n_samples, int32_t* offsets, float* t_zero, uint8_t* status, void* workspace,
                          size_t ws_bytes, int32_t reps, float* best_ms, tsdfs_stream_t stream);
int tsdfs_set_bounds_launch_shape(int32_t block, int32_t blocks_per_sm);
int tsdfs_bounds_launch_shape(int32_t* block, int32_t* blocks_per_sm);

/* ---- L2 read bandwidth (measurement support; no paper counterpart) ----
 * Streams 16-byte loads over `bytes` of the device buffer `buf` (16-byte
 * aligned; keep it well below the L2 size so it stays resident) once untimed,
 * then `reps` times between CUDA events on `stream` (synchronises it);
 * *ms_out (host) = the timed pass's milliseconds, so the achieved L2 read
 * bandwidth is reps * bytes / ms_out.  sink: a device uint32 the kernel may
 * write (keeps the loads).  The bench judges the ray march against this peak
 * when its grid stays in L2.  Returns 0 or a negative TSDFS_E_* code.        */
int tsdfs_l2_read_probe(const void* buf, size_t bytes, int32_t reps, uint32_t* sink, float* ms_out,
                        tsdfs_stream_t stream);

/* ---- which tensor-core kernel evaluates the networks (Eq. 1's MLP samples) ----
 * Both kernels compute the same per-sample quantities (SDF value and gradient,
 * colour) for render_rays and the full-evaluation passes of the samplers:
 *   TSDFS_NETKERNEL_SERIAL     64-sample tiles (four rows per sample fill both
 *                              TMEM accumulators); a layer's epilogue and the
 *                              next layer's MMAs run one after the other;
 *   TSDFS_NETKERNEL_PIPELINED  32-sample tiles, consecutive layers in alternate
 *                              halves of TMEM, so the next layer's MMAs run on
 *                              each 64-column block of its operand as soon as the
 *                              epilogue has written it.
 * The choice is process-wide, per precision (TSDFS_PREC_BF16, _F16; BF16X2 runs
 * on the pipelined kernel only and rejects SERIAL); it takes effect at the next
 * launch.  Returns 0 or TSDFS_E_INVALID.  tsdfs_network_kernel returns the
 * current choice for a precision, or TSDFS_E_INVALID.                       */
/* ---- test-only limits of the failure paths (no paper counterpart) ----
 * For tests of the device-side failure reporting without a GPU fault:
 * spin_limit (0: the default, about 6.7e7) bounds the polls of every mbarrier
 * wait of the tensor-core network kernels before the wait gives up;
 * withhold_chunk >= 0 makes their weight producers stop before that weight
 * chunk of each CTA's first tile, so the MMA issuer's wait for it runs out
 * (-1: never); march_step_cap > 0 bounds the voxel steps of a ray walk in
 * tsdf_ray_bounds (0: nx + ny + nz + 8, more than any walk takes).  A wait that
 * runs out sets TSDFS_DEV_TIMEOUT (the kernel drains its copies and MMAs, frees
 * TMEM and returns; compositing writes zeros while the status word holds it);
 * a walk cut short sets TSDFS_DEV_MARCH_CAP and ends as if it had left the
 * grid (FALLBACK over [t0, t_end] in the near phase, t_f = t_end in the far
 * phase).  Process-wide, read at each launch; 0 / -1 / 0 restores normal
 * operation.  Returns 0 or TSDFS_E_INVALID.                                 */
int tsdfs_set_test_limits(uint32_t spin_limit, int32_t march_step_cap, int32_t withhold_chunk);

#define TSDFS_NETKERNEL_SERIAL 1
#define TSDFS_NETKERNEL_PIPELINED 2
int tsdfs_set_network_kernel(int32_t precision, int32_t kernel);
int tsdfs_network_kernel(int32_t precision);
/* Set-up call: times render_rays (arguments as there, eik not written) with each
 * network kernel the precision has, reps calls each after one untimed call,
 * with CUDA events on `stream` (synchronises it), keeps the faster for
 * mlp->precision (tsdfs_set_network_kernel) and returns it (> 0), or a negative
 * code (the previous choice is then kept).  ms_out (nullable, host, 2 floats)
 * receives the mean time per call of the serial and the pipelined kernel (-1
 * for a kernel the precision does not have).  The outputs hold the last call's
 * render.                                                                   */
int tsdfs_autotune_network(const tsdfs_mlp* mlp, const float* ray_o, const float* ray_d, const float* t_n,
                           const float* t_f, const int32_t* offsets, const uint8_t* status, int64_t n_rays,
                           int64_t max_samples, float* rgb, float* depth, float* wsum, float* normal, void* ws,
                           size_t ws_bytes, int32_t reps, float* ms_out, tsdfs_stream_t stream);

/* ---- adaptive sample counts relative to the mean interval (Sec. 3.4) -------
 * Samples sit at equal spacing inside [t_n, t_f], so a ray's count is
 * proportional to its interval's length; the supplementary ray study scales it
 * against the average interval (longer than average -> more samples, shorter
 * -> fewer).  Two passes over the bounds of tsdf_ray_bounds (device arrays):
 *   mean   = FP32 of the FP64 mean of L_r = t_f[r] - t_n[r] (FP32 subtraction)
 *            over the BOUNDED rays (0 if there are none), summed in a fixed
 *            order, so repeatable;
 *   dl     = mean / n_mean (FP32, IEEE division);
 *   n[r]   = BOUNDED: clamp(ceil(L_r / dl), n_min, n_max) (FP32 division;
 *            n_min if dl == 0); FALLBACK: n_fallback; MISS: 0;
 *   offsets: exclusive scan of n, n_rays + 1 entries.
 * mean_len (device float[1]) receives the mean, or is NULL.  Requires
 * 0 < n_mean <= 4096, 1 <= n_min <= n_max <= 4096, 0 <= n_fallback <= 4096,
 * max(n_max, n_fallback) * n_rays < 2^31, else TSDFS_E_INVALID.  workspace >=
 * tsdfs_adaptive_counts_workspace_size.  Ordered on `stream`.               */
size_t tsdfs_adaptive_counts_workspace_size(int64_t n_rays);
int tsdf_adaptive_counts(const float* t_n, const float* t_f, const uint8_t* status, int64_t n_rays, float n_mean,
                         int32_t n_min, int32_t n_max, int32_t n_fallback, int32_t* n_samples, int32_t* offsets,
                         float* mean_len, void* workspace, size_t ws_bytes, tsdfs_stream_t stream);

/* ---- coarse + fine samples inside the TSDF bound (Tab. 2 "Ours", Sec. B) ---
 * The hierarchical sampler restricted to each ray's [t_n, t_f]: ray r's
 * c_r = offsets[r+1] - offsets[r] coarse midpoints of [t_n, t_f] (the counts of
 * tsdf_ray_bounds, of tsdf_adaptive_counts, or any caller's) are evaluated for
 * SDF values only; their sections give the NeuS up-sampling weights (as
 * render_rays_hier) and n_fine inverse-CDF samples at u = (k+1/2)/n_fine over
 * pdf ~ w + 1e-5; the c_r + n_fine sorted samples are evaluated fully and
 * composited with section boundaries halfway between neighbours and the outer
 * ones at t_n, t_f.  A ray with one coarse sample has no section: its fine
 * samples are the midpoints of n_fine equal parts of [t_n, t_f].  A ray with
 * no coarse sample (MISS) renders to zero.  Fixed counts over the bound are
 * the "naive" variant of Tab. 2, adaptive counts the "full" one.
 * 0 <= n_fine <= 32; max_coarse >= offsets[n_rays] (else the status word gets
 * TSDFS_DEV_SAMPLES_OVERFLOW and the outputs are zero); max_coarse +
 * n_rays * n_fine < 2^31.  Outputs as render_rays.  workspace >=
 * tsdfs_hier_bounded_workspace_size.                                        */
size_t tsdfs_hier_bounded_workspace_size(const tsdfs_mlp* mlp, int64_t n_rays, int32_t n_fine, int64_t max_coarse);
int render_rays_hier_bounded(const tsdfs_mlp* mlp, const float* ray_o, const float* ray_d, const float* t_n,
                             const float* t_f, const int32_t* offsets, const uint8_t* status, int64_t n_rays,
                             int32_t n_fine, int64_t max_coarse, float* rgb, float* depth, float* wsum, float* normal,
                             void* workspace, size_t ws_bytes, tsdfs_stream_t stream);

/* ---- backward of render_rays (training step of the networks) ---------------
 * Gradients of L = sum_r d_rgb_r . rgb_r + d_depth_r depth_r + d_eik_r eik_r
 * (the outputs of render_rays for the same inputs; eik_r is the per-ray sum
 * of (|grad f| - 1)^2 over the samples of BOUNDED rays) with respect to the
 * packed fp32 parameters, ACCUMULATED (+=) into d_sdf_w / d_rgb_w (layout of
 * sdf_w / rgb_w; the caller zeroes them).  This includes the second-order
 * terms through grad f (opacity, colour-network normal, eikonal).  d_rgb:
 * [n_rays][3]; d_depth, d_eik: [n_rays] or NULL (zero).  FP32 parameters and
 * arithmetic (mlp->precision is ignored).  Two implementations, chosen
 * process-wide by tsdfs_set_backward_kernel:
 *  - TSDFS_BACKWARD_GEMM (default): layer-major.  Each layer of both networks
 *    is a GEMM over a chunk of samples (4 rows per sample for the SDF
 *    network: the value and its three x-derivative rows) on the tensor cores,
 *    FP32 operands emulated by three BF16 parts (cuBLAS BF16x9, FP32
 *    accumulation, the emulation's handling of infinite and NaN operands
 *    off: non-finite parameters set TSDFS_DEV_NONFINITE instead); the
 *    element-wise steps are the library's kernels.  The call reads the sample
 *    total offsets[n_rays] from the device first (one synchronisation of
 *    `stream`).  The workspace holds the per-sample records
 *    and the activations of one chunk (tsdfs_set_backward_chunk; by default as
 *    many samples as fit 16 GiB, at most max_samples); a batch larger than one
 *    chunk recomputes each chunk's activations once more.  The first call on
 *    a device creates the library's cuBLAS handle (cuBLAS allocates its own
 *    state then); the GEMMs' workspace is taken from `workspace`.
 *  - TSDFS_BACKWARD_SIMT: FP32 SIMT; activations recomputed per tile of 8
 *    samples; the workspace is the per-sample records plus a per-SM scratch
 *    and a private gradient copy per block.  Fully asynchronous.
 * workspace >= tsdfs_backward_workspace_size, which sizes it for the current
 * choice of implementation and chunk.                                       */
#define TSDFS_BACKWARD_SIMT 1
#define TSDFS_BACKWARD_GEMM 2
/* Choose the implementation of render_rays_backward (process-wide).  Returns 0
 * or TSDFS_E_INVALID.  tsdfs_backward_kernel returns the current choice.     */
int tsdfs_set_backward_kernel(int32_t kind);
int32_t tsdfs_backward_kernel(void);
/* Samples per chunk of the layer-major backward (0: as many as fit 16 GiB of
 * activations).  Smaller chunks need less workspace and recompute the
 * forward once more.  Returns 0 or TSDFS_E_INVALID (negative, or 2^29
 * samples or more).                                                         */
int tsdfs_set_backward_chunk(int64_t samples);
/* Samples per chunk the layer-major backward uses for this network and
 * max_samples (>= 1) under the current chunk setting; a batch of more samples
 * runs in several chunks.  Returns the count or TSDFS_E_INVALID.            */
int64_t tsdfs_backward_chunk_samples(const tsdfs_mlp* mlp, int64_t max_samples);
size_t tsdfs_backward_workspace_size(const tsdfs_mlp* mlp, int64_t n_rays, int64_t max_samples);
int render_rays_backward(const tsdfs_mlp* mlp, const float* ray_o, const float* ray_d, const float* t_n,
                         const float* t_f, const int32_t* offsets, const uint8_t* status, int64_t n_rays,
                         int64_t max_samples, const float* d_rgb, const float* d_depth, const float* d_eik,
                         float* d_sdf_w, float* d_rgb_w, void* workspace, size_t ws_bytes, tsdfs_stream_t stream);

/* ---- training step: a forward that keeps what the backward needs -----------
 * render_rays_train: render_rays with FP32 networks evaluated by the
 * layer-major path of render_rays_backward (every layer a GEMM over a chunk of
 * samples, FP32 operands emulated by BF16 parts on the tensor cores); same
 * outputs as render_rays.  It leaves the per-sample records and the last
 * chunk's activations (all of them when the batch fits one chunk) in
 * `workspace`.  render_rays_backward_kept, called next with the same mlp
 * parameters, rays, bounds, max_samples and workspace (none of them changed in
 * between), returns the gradients of render_rays_backward without
 * recomputing what was kept.  Both read the sample total offsets[n_rays] from
 * the device (one synchronisation of `stream`).  workspace >=
 * tsdfs_train_workspace_size: the layer-major backward's workspace, whatever
 * tsdfs_set_backward_kernel chose.  mlp->precision is ignored (FP32).  The
 * paper trains its networks (Sec. 4.2) but prescribes no such split; it is
 * the training step of this library's render path.                           */
size_t tsdfs_train_workspace_size(const tsdfs_mlp* mlp, int64_t n_rays, int64_t max_samples);
int render_rays_train(const tsdfs_mlp* mlp, const float* ray_o, const float* ray_d, const float* t_n,
                      const float* t_f, const int32_t* offsets, const uint8_t* status, int64_t n_rays,
                      int64_t max_samples, float* rgb, float* depth, float* wsum, float* normal, float* eik,
                      void* workspace, size_t ws_bytes, tsdfs_stream_t stream);
int render_rays_backward_kept(const tsdfs_mlp* mlp, const float* ray_o, const float* ray_d, const float* t_n,
                              const float* t_f, const int32_t* offsets, const uint8_t* status, int64_t n_rays,
                              int64_t max_samples, const float* d_rgb, const float* d_depth, const float* d_eik,
                              float* d_sdf_w, float* d_rgb_w, void* workspace, size_t ws_bytes,
                              tsdfs_stream_t stream);

/* ---- BF16 tensor-core parameter layout --------------------------------------
 * tsdfs_pack_mlp converts sdf_w / rgb_w to the 16-bit K-major tiles the
 * tcgen05 path reads -- bf16, or fp16 when mlp->precision is TSDFS_PREC_F16 --
 * rounded to nearest even, into `packed` (device, tsdfs_packed_size bytes,
 * 16-byte aligned).  Repeat after every parameter update.  Layout: every
 * layer of both networks in order, each padded to 16 rows and columns and cut
 * into 64-column chunks of 8x8 core matrices; then the serial kernel's two
 * folded layers (the SDF output layer's value row net_0, and the first colour
 * layer applied to [h, x~, direction encoding, unit normal] with h the last
 * hidden SDF activation: weights [W_c,feat W_f | W_c,x | W_c,dir | W_c,n],
 * the product summed in FP32 and then rounded), and their FP32 biases
 * (b_f,0, and b_c + W_c,feat b_f), 16-byte aligned.  The folding is exact in
 * real arithmetic: the features enter the colour network linearly.          */
/* ---- FP64 finite-difference harness of render_rays_backward (test use) ----
 * The bounded render of render_rays (same inputs: rays, [t_n, t_f], offsets,
 * status; midpoint samples; both networks with the SDF gradient; the network's
 * opacity; Eq. 1 / Eq. 2) evaluated in FP64 on the GPU with FP64 parameters
 * sdf_w64 / rgb_w64 (device, the packed (W, b) layout of tsdfs_sdf_param_count /
 * tsdfs_rgb_param_count doubles; mlp supplies the architecture, constants and
 * opacity, its own parameter pointers are not read), reduced to
 *   *loss = sum_r g_rgb[r] . rgb[r] + g_depth[r] depth[r] + g_eik[r] eik[r]
 * (g_depth, g_eik nullable; eik as in render_rays: BOUNDED rays only), the
 * functional whose parameter gradient render_rays_backward returns for output
 * gradients g_rgb, g_depth, g_eik.  Central differences of *loss over single
 * parameters check that gradient.  The one use of FP64 arithmetic on the GPU;
 * it synchronises `stream` once to read the sample total.  loss is a device
 * double; ws >= tsdfs_loss_f64_workspace_size(n_rays, max_samples) (about 20 KB
 * per sample).  Returns 0 or a negative TSDFS_E_* code.                     */
size_t tsdfs_loss_f64_workspace_size(int64_t n_rays, int64_t max_samples);
int tsdfs_loss_f64(const tsdfs_mlp* mlp, const double* sdf_w64, const double* rgb_w64, const float* ray_o,
                   const float* ray_d, const float* t_n, const float* t_f, const int32_t* offsets,
                   const uint8_t* status, int64_t n_rays, int64_t max_samples, const float* g_rgb,
                   const float* g_depth, const float* g_eik, double* loss, void* ws, size_t ws_bytes,
                   tsdfs_stream_t stream);

size_t tsdfs_packed_size(int32_t arch);
int tsdfs_pack_mlp(const tsdfs_mlp* mlp, void* packed, tsdfs_stream_t stream);

/* ---- parameter check (failure detection; no counterpart in the paper) --------
 * Scans sdf_w and rgb_w (device, fp32) and sets TSDFS_DEV_NONFINITE in the
 * status word (tsdfs_sync_status) if any parameter is NaN or infinite;
 * tsdfs_pack_mlp sets the same bit for the values it packs.  Nothing traps.  */
int tsdfs_check_mlp(const tsdfs_mlp* mlp, tsdfs_stream_t stream);

/* ---- kernel timing (instrumentation; no counterpart in the paper) ------------
 * tsdfs_profile(1) clears the record and starts timing: every kernel launch
 * of the library is then bracketed by two CUDA events recorded on its launch
 * stream; tsdfs_profile(0) stops and clears.  tsdfs_profile_read synchronises
 * the recorded events and returns, for launches whose kernel name starts with
 * `prefix` ("" = all), the summed device time in ms and the launch count.   */
int tsdfs_profile(int32_t enable);
int tsdfs_profile_read(const char* prefix, double* total_ms, int64_t* launches);

/* sizes of the packed fp32 parameter arrays, in floats */
int64_t tsdfs_sdf_param_count(int32_t arch);
int64_t tsdfs_rgb_param_count(int32_t arch);

#ifdef __cplusplus
}
#endif
#endif /* TSDFS_H */
