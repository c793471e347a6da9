// Backward of render_rays: parameter gradients of
//   L = sum_r d_rgb_r . rgb_r + d_depth_r depth_r + d_eik_r eik_r.
//
// Two paths share the first two steps:
// 1. a forward network pass recomputes the per-sample records;
// 2. k_comp_bwd (one thread per ray) differentiates the compositing of Eq. 1,
//    Eq. 2 and the NeuS opacity, and adds the eikonal term: per-sample adjoints
//    of f, grad f and the colour.
// The layer-major path (backward_gemm.cu, the default) then runs each layer of
// both networks as GEMMs over a chunk of samples on the tensor cores.  The SIMT
// path of this file:
// 3. k_mlp_bwd (FP32 SIMT, tiles of kTB samples) recomputes both networks with
//    their forward-mode tangent rows into a per-block scratch, then
//    back-propagates values and tangents (the slope sigma(beta z) of a hidden
//    layer is differentiated too: d slope / dz = beta sigma (1 - sigma)), and
//    accumulates parameter gradients into a private copy per block;
// 4. k_reduce_grads adds the private copies into the caller's gradients.
#include <atomic>

#include "backward.cuh"

namespace tsdfs {

template <int ARCH>
int launch_mlp_full_simt(const NetParams& np, const SampleSource& src, SampleRec* rec, int64_t max_samples,
                         cudaStream_t st);

namespace {

constexpr int kBThreads = 256;
constexpr int kTB = 8;                // samples per tile
constexpr int kRows = 4 * kTB;        // SDF rows (value + 3 tangents per sample)
constexpr int kLD = 292;              // row stride of the shared buffers (>= 289 + pad)
constexpr int kKC = 16;

__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + expf(-x)); }

// ---- 2. compositing backward ------------------------------------------------
__global__ void k_comp_bwd(const SampleRec* __restrict__ rec, const int32_t* __restrict__ offsets,
                           const uint8_t* __restrict__ status, const float* __restrict__ ray_d, int64_t n_rays,
                           Opacity op, const float* __restrict__ d_rgb, const float* __restrict__ d_depth,
                           const float* __restrict__ d_eik, SampleAdj* __restrict__ adj) {
    const float kClamp = 1.0f - 5.9604645e-8f;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rays; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = offsets[r], e = offsets[r + 1];
        const bool bounded = status[r] == TSDFS_BOUNDED;
        const float dr = d_rgb[3 * r], dg = d_rgb[3 * r + 1], db = d_rgb[3 * r + 2];
        const float dd_r = d_depth ? d_depth[r] : 0.0f;
        const float de_r = d_eik ? d_eik[r] : 0.0f;
        const float v[3] = {ray_d[3 * r], ray_d[3 * r + 1], ray_d[3 * r + 2]};
        const float inv_s = op.inv_s, eps = op.eps;
        const bool volsdf = op.kind == TSDFS_OPACITY_VOLSDF;
        // NeuS: plo / phi = Phi at the section ends, araw = the unclamped ratio;
        // VolSDF: plo = the density, phi = exp(-density * delta) = 1 - alpha, araw = alpha
        auto alpha_of = [&](const SampleRec& R, float& plo, float& phi, float& araw) {
            if (volsdf) {
                plo = laplace_density(R.f, inv_s);
                phi = expf(-plo * R.delta);
                araw = -expm1f(-plo * R.delta);
                return araw;
            }
            const float c = fminf(R.dd, 0.0f);
            plo = sigm(inv_s * (R.f - 0.5f * R.delta * c));
            phi = sigm(inv_s * (R.f + 0.5f * R.delta * c));
            araw = (plo - phi + eps) / (plo + eps);
            return fminf(fmaxf(araw, 0.0f), 1.0f);
        };
        // pass 1: totals
        float logT = 0.0f, W = 0.0f, D = 0.0f;
        for (int64_t g = b; g < e; ++g) {
            float plo, phi, araw;
            const float a = alpha_of(rec[g], plo, phi, araw);
            const float w = expf(logT) * a;
            W += w;
            D += w * rec[g].t;
            logT += log1pf(-fminf(a, kClamp));
        }
        const bool okW = W >= 1e-8f;
        const float depth = okW ? D / W : 0.0f;
        const float invW = okW ? 1.0f / W : 0.0f;
        // pass 2: G = sum_k dL/dw_k w_k
        float G = 0.0f;
        logT = 0.0f;
        for (int64_t g = b; g < e; ++g) {
            const SampleRec& R = rec[g];
            float plo, phi, araw;
            const float a = alpha_of(R, plo, phi, araw);
            const float w = expf(logT) * a;
            const float gw = dr * R.r + dg * R.g + db * R.b + (okW ? dd_r * (R.t - depth) * invW : 0.0f);
            G += gw * w;
            logT += log1pf(-fminf(a, kClamp));
        }
        // pass 3: per-sample adjoints
        float P = 0.0f;
        logT = 0.0f;
        for (int64_t g = b; g < e; ++g) {
            const SampleRec& R = rec[g];
            float plo, phi, araw;
            const float a = alpha_of(R, plo, phi, araw);
            const float T = expf(logT);
            const float w = T * a;
            const float gw = dr * R.r + dg * R.g + db * R.b + (okW ? dd_r * (R.t - depth) * invW : 0.0f);
            P += gw * w;
            const float S = G - P;  // sum over later samples of dL/dw_k w_k
            const float dlt = a < kClamp ? -1.0f / (1.0f - a) : 0.0f;
            const float ga = gw * T + S * dlt;
            float gf, gdd;
            if (volsdf) {
                // d alpha / d f = exp(-sigma delta) delta d sigma / d f
                gf = ga * phi * R.delta * laplace_density_slope(R.f, inv_s);
                gdd = 0.0f;
            } else {
                const float ga_raw = (araw > 0.0f && araw < 1.0f) ? ga : 0.0f;
                const float Dn = plo + eps;
                const float g_plo = ga_raw * phi / (Dn * Dn);
                const float g_phi = -ga_raw / Dn;
                const float g_xlo = g_plo * inv_s * plo * (1.0f - plo);
                const float g_xhi = g_phi * inv_s * phi * (1.0f - phi);
                gf = g_xlo + g_xhi;
                const float gc = 0.5f * R.delta * (g_xhi - g_xlo);
                gdd = R.dd < 0.0f ? gc : 0.0f;
            }
            float ggx = gdd * v[0], ggy = gdd * v[1], ggz = gdd * v[2];
            if (bounded && de_r != 0.0f) {
                // d/dg of (|g| - 1)^2 = 2 (|g| - 1) g / |g| = 2 (|g| - 1) n^
                const float k = 2.0f * de_r * (R.gnorm - 1.0f);
                ggx += k * R.nx;
                ggy += k * R.ny;
                ggz += k * R.nz;
            }
            SampleAdj A;
            A.gf = gf; A.ggx = ggx; A.ggy = ggy; A.ggz = ggz;
            A.gr = w * dr; A.gg = w * dg; A.gb = w * db; A.pad = 0.0f;
            adj[g] = A;
            logT += log1pf(-fminf(a, kClamp));
        }
    }
}

// ---- 3. network backward ------------------------------------------------------
struct BwdSmem {
    float a[kRows][kLD];    // layer input (forward) / adjoint of the layer input (backward)
    float b[kRows][kLD];    // layer pre-activation (forward) / its adjoint (backward)
    float c[kRows][kLD];    // scratch
    float wt[kKC][kLD];     // weight chunk
    float xt[kTB][3], dir[kTB][3], nh[kTB][3], gn[kTB];
    float adj[kTB][8];
    int valid[kTB];
};

struct BwdParams {
    NetParams np;
    SampleSource src;
    const SampleAdj* adj;
    const SampleRec* rec;
    float* scratch;     // per block: activations of one tile
    int64_t scratch_floats;
    float* gcopy;       // per block: private gradient copy (sdf params then rgb params)
    int64_t gcopy_floats;
};

// out[r][n] = sum_k in[r][k] W[n][k] (+ b[n] on bias rows) for r < R, n < N
template <int R>
__device__ void fwd_gemm(BwdSmem& sm, const float (*in)[kLD], int K, const float* __restrict__ W, int N,
                         const float* __restrict__ bias, bool bias_all_rows, float (*out)[kLD]) {
    const int tid = threadIdx.x;
    for (int n0 = 0; n0 < N; n0 += kBThreads / (R <= 8 ? 1 : 1)) {
        const int n = n0 + tid;
        float acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = 0.0f;
        for (int k0 = 0; k0 < K; k0 += kKC) {
            __syncthreads();
            for (int e = tid; e < kKC * kBThreads; e += kBThreads) {
                const int kk = e % kKC, nn = n0 + e / kKC;
                sm.wt[kk][nn - n0] = (nn < N && k0 + kk < K) ? __ldg(W + (int64_t)nn * K + k0 + kk) : 0.0f;
            }
            __syncthreads();
            const int km = K - k0 < kKC ? K - k0 : kKC;
            for (int kk = 0; kk < km; ++kk) {
                const float w = sm.wt[kk][tid];
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] = fmaf(in[r][k0 + kk], w, acc[r]);
            }
        }
        __syncthreads();
        if (n < N) {
            const float bb = __ldg(bias + n);
#pragma unroll
            for (int r = 0; r < R; ++r) out[r][n] = acc[r] + ((bias_all_rows || (r & 3) == 0) ? bb : 0.0f);
        }
    }
    __syncthreads();
}

// gin[r][k] = sum_n g[r][n] W[n][k] for r < R, k < K
template <int R>
__device__ void bwd_gemm(BwdSmem& sm, const float (*g)[kLD], int N, const float* __restrict__ W, int K,
                         float (*gin)[kLD]) {
    const int tid = threadIdx.x;
    for (int k0 = 0; k0 < K; k0 += kBThreads) {
        const int k = k0 + tid;
        float acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = 0.0f;
        for (int nc = 0; nc < N; nc += kKC) {
            __syncthreads();
            for (int e = tid; e < kKC * kBThreads; e += kBThreads) {
                const int nn = nc + e / kBThreads, kk = k0 + e % kBThreads;
                sm.wt[e / kBThreads][e % kBThreads] = (nn < N && kk < K) ? __ldg(W + (int64_t)nn * K + kk) : 0.0f;
            }
            __syncthreads();
            const int nm = N - nc < kKC ? N - nc : kKC;
            for (int j = 0; j < nm; ++j) {
                const float w = sm.wt[j][tid];
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] = fmaf(g[r][nc + j], w, acc[r]);
            }
        }
        __syncthreads();
        if (k < K) {
#pragma unroll
            for (int r = 0; r < R; ++r) gin[r][k] = acc[r];
        }
    }
    __syncthreads();
}

// dW[n][k] += sum_r g[r][n] in[r][k]; db[n] += sum over bias rows of g[r][n]
template <int R>
__device__ void grad_accum(const float (*g)[kLD], const float (*in)[kLD], int N, int K, float* __restrict__ dW,
                           float* __restrict__ db, bool bias_all_rows) {
    const int tid = threadIdx.x;
    for (int64_t e = tid; e < (int64_t)N * K; e += kBThreads) {
        const int n = (int)(e / K), k = (int)(e % K);
        float s = 0.0f;
#pragma unroll
        for (int r = 0; r < R; ++r) s = fmaf(g[r][n], in[r][k], s);
        dW[e] += s;
    }
    for (int n = tid; n < N; n += kBThreads) {
        float s = 0.0f;
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (bias_all_rows || (r & 3) == 0) s += g[r][n];
        db[n] += s;
    }
    __syncthreads();
}

__device__ __forceinline__ float enc_val_b(const float* xt, int j, int pe, int a, bool deriv) {
    if (j < 3) return deriv ? (j == a ? 1.0f : 0.0f) : xt[j];
    const int q = j - 3;
    const int oct = q / 6, part = (q % 6) / 3, b = q % 3;
    if (oct >= pe) return 0.0f;
    if (deriv && b != a) return 0.0f;
    const float f = (float)(1 << oct);
    float sn, cs;
    sincosf(f * xt[b], &sn, &cs);
    if (!deriv) return part == 0 ? sn : cs;
    return part == 0 ? f * cs : -f * sn;
}

template <int ARCH>
__global__ void __launch_bounds__(kBThreads, 1) k_mlp_bwd(BwdParams p) {
    using A = Arch<ARCH>;
    constexpr int LS = A::kSdfLayers, LC = A::kRgbLayers;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdSmem& sm = *reinterpret_cast<BwdSmem*>(smem_raw);
    const int tid = threadIdx.x;
    const float beta = p.np.beta;
    float* scr = p.scratch + blockIdx.x * p.scratch_floats;
    float* gsdf = p.gcopy + blockIdx.x * p.gcopy_floats;
    float* grgb = gsdf + sdf_param_count<ARCH>();
    const int64_t total = (int64_t)__ldg(p.src.total_dev);
    if (total > p.src.capacity) return;
    const int64_t n_tiles = (total + kTB - 1) / kTB;
    // scratch layout: for each SDF layer l: In_l [kRows][K_l] then Pre_l [kRows][N_l];
    // then for each colour layer: In [kTB][K] then Pre [kTB][N]
    auto sdf_in = [&](int l) {
        int64_t o = 0;
        for (int i = 0; i < l; ++i) o += (int64_t)kRows * (A::sdf(i).in + A::sdf(i).out);
        return scr + o;
    };
    auto sdf_pre = [&](int l) { return sdf_in(l) + (int64_t)kRows * A::sdf(l).in; };
    auto rgb_in = [&](int l) {
        int64_t o = 0;
        for (int i = 0; i < LS; ++i) o += (int64_t)kRows * (A::sdf(i).in + A::sdf(i).out);
        for (int i = 0; i < l; ++i) o += (int64_t)kTB * (A::rgb(i).in + A::rgb(i).out);
        return scr + o;
    };
    auto rgb_pre = [&](int l) { return rgb_in(l) + (int64_t)kTB * A::rgb(l).in; };
    auto save = [&](float* dst, const float (*src)[kLD], int R, int n) {
        for (int e = tid; e < R * n; e += kBThreads) dst[e] = src[e / n][e % n];
    };
    auto load = [&](float (*dst)[kLD], const float* src, int R, int n) {
        for (int e = tid; e < R * n; e += kBThreads) dst[e / n][e % n] = src[e];
    };

    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        __syncthreads();
        if (tid < kTB) {
            const int s = tid;
            const int64_t g = tile * kTB + s;
            const bool ok = g < total;
            int64_t r = 0;
            float t = 0.0f;
            if (ok) {
                r = find_ray(p.src.offsets, p.src.n_rays, g);
                t = p.rec[g].t;
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float o = ok ? __ldg(p.src.ray_o + 3 * r + a) : 0.0f;
                const float d = ok ? __ldg(p.src.ray_d + 3 * r + a) : 0.0f;
                sm.dir[s][a] = d;
                sm.xt[s][a] = (o + t * d - p.np.center[a]) * p.np.inv_scale;
            }
            const float4* A4 = reinterpret_cast<const float4*>(p.adj + (ok ? g : 0));
            const float4 a0 = ok ? A4[0] : make_float4(0, 0, 0, 0), a1 = ok ? A4[1] : make_float4(0, 0, 0, 0);
            sm.adj[s][0] = a0.x; sm.adj[s][1] = a0.y; sm.adj[s][2] = a0.z; sm.adj[s][3] = a0.w;
            sm.adj[s][4] = a1.x; sm.adj[s][5] = a1.y; sm.adj[s][6] = a1.z; sm.adj[s][7] = 0.0f;
            sm.valid[s] = ok;
        }
        __syncthreads();
        // ---- SDF forward with tangents (row 4s + c: c = 0 value, 1..3 d/dx, d/dy, d/dz) ----
        for (int e = tid; e < kRows * A::kEnc; e += kBThreads) {
            const int row = e / A::kEnc, k = e % A::kEnc;
            const int s = row >> 2, c = row & 3;
            sm.a[row][k] = c == 0 ? enc_val_b(sm.xt[s], k, A::kPeSdf, 0, false)
                                  : enc_val_b(sm.xt[s], k, A::kPeSdf, c - 1, true);
        }
        __syncthreads();
        for (int l = 0; l < LS; ++l) {
            const Layer ly = A::sdf(l);
            const float* W = p.np.sdf_w + sdf_layer_offset<ARCH>(l);
            const float* bb = W + (int64_t)ly.out * ly.in;
            save(sdf_in(l), sm.a, kRows, ly.in);
            fwd_gemm<kRows>(sm, sm.a, ly.in, W, ly.out, bb, false, sm.b);
            save(sdf_pre(l), sm.b, kRows, ly.out);
            if (l == LS - 1) break;
            // activation -> next input (skip concat before layer kSkip)
            const bool skip_next = l + 1 == A::kSkip;
            const float sc = skip_next ? 0.70710678118654752f : 1.0f;
            for (int e = tid; e < kRows * ly.out; e += kBThreads) {
                const int row = e / ly.out, n = e % ly.out;
                const int vrow = row & ~3;
                const float z = sm.b[vrow][n];
                const float bz = beta * z;
                float v;
                if ((row & 3) == 0) v = bz > 20.0f ? z : log1pf(expf(bz)) / beta;
                else v = (bz > 20.0f ? 1.0f : 1.0f / (1.0f + expf(-bz))) * sm.b[row][n];
                sm.c[row][n] = v * sc;
            }
            __syncthreads();
            if (skip_next) {
                const int hw = ly.out;
                for (int e = tid; e < kRows * A::kEnc; e += kBThreads) {
                    const int row = e / A::kEnc, k = e % A::kEnc;
                    const int s = row >> 2, c = row & 3;
                    sm.c[row][hw + k] = sc * (c == 0 ? enc_val_b(sm.xt[s], k, A::kPeSdf, 0, false)
                                                     : enc_val_b(sm.xt[s], k, A::kPeSdf, c - 1, true));
                }
            }
            __syncthreads();
            for (int e = tid; e < kRows * A::sdf(l + 1).in; e += kBThreads) sm.a[e / A::sdf(l + 1).in][e % A::sdf(l + 1).in] =
                sm.c[e / A::sdf(l + 1).in][e % A::sdf(l + 1).in];
            __syncthreads();
        }
        // sm.b holds the SDF output rows: value row [net0, feature], tangent rows [d net0, ...]
        if (tid < kTB) {
            const int s = tid;
            const float gx = sm.b[4 * s + 1][0], gy = sm.b[4 * s + 2][0], gz = sm.b[4 * s + 3][0];
            const float g = sqrtf(gx * gx + gy * gy + gz * gz);
            const float inv = g > 0.0f ? 1.0f / g : 0.0f;
            sm.nh[s][0] = gx * inv; sm.nh[s][1] = gy * inv; sm.nh[s][2] = gz * inv;
            sm.gn[s] = g;
        }
        __syncthreads();
        // colour input rows (one per sample) into sm.c rows 0..kTB-1
        {
            constexpr int kDir = A::kDirEnc, kFeatCol = 3 + kDir + 3;
            const int Kc = A::rgb(0).in;
            for (int e = tid; e < kTB * Kc; e += kBThreads) {
                const int s = e / Kc, col = e % Kc;
                float v;
                if (col < 3) v = sm.xt[s][col];
                else if (col < 3 + kDir) v = A::kPeDir == 0 ? sm.dir[s][col - 3] : enc_val_b(sm.dir[s], col - 3, A::kPeDir, 0, false);
                else if (col < kFeatCol) v = sm.nh[s][col - 3 - kDir];
                else v = sm.b[4 * s][col - kFeatCol + 1];
                sm.c[s][col] = v;
            }
        }
        __syncthreads();
        // ---- colour forward ----
        for (int l = 0; l < LC; ++l) {
            const Layer ly = A::rgb(l);
            const float* W = p.np.rgb_w + rgb_layer_offset<ARCH>(l);
            const float* bb = W + (int64_t)ly.out * ly.in;
            save(rgb_in(l), sm.c, kTB, ly.in);
            fwd_gemm<kTB>(sm, sm.c, ly.in, W, ly.out, bb, true, sm.a);
            save(rgb_pre(l), sm.a, kTB, ly.out);
            if (l == LC - 1) break;
            for (int e = tid; e < kTB * ly.out; e += kBThreads) sm.c[e / ly.out][e % ly.out] = fmaxf(sm.a[e / ly.out][e % ly.out], 0.0f);
            __syncthreads();
        }
        // ---- colour backward: g(pre) of the output = g(rgb) * rgb (1 - rgb) ----
        for (int e = tid; e < kTB * 3; e += kBThreads) {
            const int s = e / 3, ch = e % 3;
            const float y = 1.0f / (1.0f + expf(-sm.a[s][ch]));
            sm.b[s][ch] = sm.valid[s] ? sm.adj[s][4 + ch] * y * (1.0f - y) : 0.0f;
        }
        __syncthreads();
        for (int l = LC - 1; l >= 0; --l) {
            const Layer ly = A::rgb(l);
            const float* W = p.np.rgb_w + rgb_layer_offset<ARCH>(l);
            load(sm.c, rgb_in(l), kTB, ly.in);
            __syncthreads();
            grad_accum<kTB>(sm.b, sm.c, ly.out, ly.in, grgb + rgb_layer_offset<ARCH>(l),
                            grgb + rgb_layer_offset<ARCH>(l) + (int64_t)ly.out * ly.in, true);
            bwd_gemm<kTB>(sm, sm.b, ly.out, W, ly.in, sm.a);
            if (l == 0) break;
            // through the ReLU of layer l - 1: pre-activation of layer l - 1 = its saved pre
            const Layer lp = A::rgb(l - 1);
            load(sm.c, rgb_pre(l - 1), kTB, lp.out);
            __syncthreads();
            for (int e = tid; e < kTB * lp.out; e += kBThreads) {
                const int s = e / lp.out, n = e % lp.out;
                sm.b[s][n] = sm.c[s][n] > 0.0f ? sm.a[s][n] : 0.0f;
            }
            __syncthreads();
        }
        // sm.a rows 0..kTB-1 = adjoint of the colour input: [x~, dir, n^, feature]
        // ---- SDF output layer adjoint ----
        {
            constexpr int kDir = A::kDirEnc, kFeatCol = 3 + kDir + 3;
            const int No = A::sdf(LS - 1).out;
            // copy the colour-input adjoint aside (sm.a is reused): rows kTB.. of sm.c
            for (int e = tid; e < kRows * No; e += kBThreads) {
                const int row = e / No, n = e % No;
                const int s = row >> 2, c = row & 3;
                float v = 0.0f;
                if (sm.valid[s]) {
                    if (c == 0) v = n == 0 ? sm.adj[s][0] * p.np.scale : sm.a[s][kFeatCol + n - 1];
                    else if (n == 0) {
                        // adjoint of grad f component c-1: compositing + eikonal + normal
                        const float g = sm.gn[s];
                        const float* nh = sm.nh[s];
                        const float gn0 = sm.a[s][3 + kDir], gn1 = sm.a[s][3 + kDir + 1], gn2 = sm.a[s][3 + kDir + 2];
                        const float dot = nh[0] * gn0 + nh[1] * gn1 + nh[2] * gn2;
                        const float gnc = c == 1 ? gn0 : (c == 2 ? gn1 : gn2);
                        const float from_n = g > 0.0f ? (gnc - nh[c - 1] * dot) / g : 0.0f;
                        v = sm.adj[s][c] + from_n;
                    }
                }
                sm.b[row][n] = v;
            }
        }
        __syncthreads();
        // ---- SDF backward ----
        for (int l = LS - 1; l >= 0; --l) {
            const Layer ly = A::sdf(l);
            const float* W = p.np.sdf_w + sdf_layer_offset<ARCH>(l);
            // sm.b = adjoint of this layer's pre-activation rows
            load(sm.c, sdf_in(l), kRows, ly.in);
            __syncthreads();
            grad_accum<kRows>(sm.b, sm.c, ly.out, ly.in, gsdf + sdf_layer_offset<ARCH>(l),
                              gsdf + sdf_layer_offset<ARCH>(l) + (int64_t)ly.out * ly.in, false);
            if (l == 0) break;
            bwd_gemm<kRows>(sm, sm.b, ly.out, W, ly.in, sm.a);   // adjoint of this layer's input
            // the input of layer l is the activation of layer l-1 (scaled and concatenated at the skip)
            const Layer lp = A::sdf(l - 1);
            const float sc = l == A::kSkip ? 0.70710678118654752f : 1.0f;
            load(sm.c, sdf_pre(l - 1), kRows, lp.out);
            __syncthreads();
            for (int e = tid; e < kRows * lp.out; e += kBThreads) {
                const int row = e / lp.out, n = e % lp.out;
                const int vrow = row & ~3;
                const float z = sm.c[vrow][n];
                const float bz = beta * z;
                const float sg = bz > 20.0f ? 1.0f : 1.0f / (1.0f + expf(-bz));
                const float dsg = bz > 20.0f ? 0.0f : beta * sg * (1.0f - sg);
                float v;
                if ((row & 3) == 0) {
                    // value row: d/dz of h (slope) and of the tangents sg * dz_a (dsg * dz_a)
                    v = sm.a[row][n] * sc * sg;
                    for (int a = 1; a <= 3; ++a) v += sm.a[row + a][n] * sc * dsg * sm.c[row + a][n];
                } else {
                    v = sm.a[row][n] * sc * sg;
                }
                sm.b[row][n] = v;
            }
            __syncthreads();
        }
    }
}

__global__ void k_zero(float* p, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = 0.0f;
}

__global__ void k_reduce_grads(const float* __restrict__ copies, int nb, int64_t per, int64_t n_sdf,
                               float* __restrict__ d_sdf, float* __restrict__ d_rgb) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < per; i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int b = 0; b < nb; ++b) s += copies[(int64_t)b * per + i];
        if (i < n_sdf) d_sdf[i] += s;
        else d_rgb[i - n_sdf] += s;
    }
}

int bwd_blocks() {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

template <int ARCH>
int64_t scratch_floats() {
    using A = Arch<ARCH>;
    int64_t o = 0;
    for (int i = 0; i < A::kSdfLayers; ++i) o += (int64_t)kRows * (A::sdf(i).in + A::sdf(i).out);
    for (int i = 0; i < A::kRgbLayers; ++i) o += (int64_t)kTB * (A::rgb(i).in + A::rgb(i).out);
    return (o + 63) / 64 * 64;
}

struct BwdWs {
    SampleRec* rec;
    SampleAdj* adj;
    float* scratch;
    float* gcopy;
    size_t bytes;
};

BwdWs bwd_layout(void* base, int arch, int64_t max_samples, int blocks) {
    BwdWs w{};
    uintptr_t p = (reinterpret_cast<uintptr_t>(base) + 255) & ~uintptr_t(255);
    auto take = [&](size_t bytes) {
        uintptr_t q = p;
        p = (p + bytes + 255) & ~uintptr_t(255);
        return q;
    };
    const int64_t sf = arch == TSDFS_ARCH_TINY ? scratch_floats<TSDFS_ARCH_TINY>() : scratch_floats<TSDFS_ARCH_ROOM>();
    const int64_t gf = arch == TSDFS_ARCH_TINY ? sdf_param_count<TSDFS_ARCH_TINY>() + rgb_param_count<TSDFS_ARCH_TINY>()
                                               : sdf_param_count<TSDFS_ARCH_ROOM>() + rgb_param_count<TSDFS_ARCH_ROOM>();
    w.rec = reinterpret_cast<SampleRec*>(take((size_t)max_samples * sizeof(SampleRec)));
    w.adj = reinterpret_cast<SampleAdj*>(take((size_t)max_samples * sizeof(SampleAdj)));
    w.scratch = reinterpret_cast<float*>(take((size_t)blocks * sf * 4));
    w.gcopy = reinterpret_cast<float*>(take((size_t)blocks * gf * 4));
    w.bytes = p - reinterpret_cast<uintptr_t>(base) + 256;
    return w;
}

std::atomic<int> g_bwd_kind{TSDFS_BACKWARD_GEMM};
std::atomic<int64_t> g_bwd_chunk{0};

}  // namespace

int launch_comp_bwd(const SampleRec* rec, const int32_t* offsets, const uint8_t* status, const float* ray_d,
                    int64_t n_rays, const tsdfs_mlp* mlp, const float* d_rgb, const float* d_depth,
                    const float* d_eik, SampleAdj* adj, cudaStream_t st) {
    k_comp_bwd<<<grid_1d(n_rays, 128), 128, 0, st>>>(rec, offsets, status, ray_d, n_rays,
                                                     Opacity{mlp->opacity, mlp->inv_s, mlp->alpha_eps}, d_rgb, d_depth,
                                                     d_eik, adj);
    return cuda_check(cudaGetLastError(), "backward composite launch");
}

int64_t backward_chunk_setting() { return g_bwd_chunk.load(); }

}  // namespace tsdfs

using namespace tsdfs;

extern "C" int tsdfs_set_backward_kernel(int32_t kind) {
    if (kind != TSDFS_BACKWARD_SIMT && kind != TSDFS_BACKWARD_GEMM) return fail(TSDFS_E_INVALID, "unknown backward kind %d", kind);
    g_bwd_kind.store(kind);
    return TSDFS_OK;
}

extern "C" int32_t tsdfs_backward_kernel(void) { return g_bwd_kind.load(); }

extern "C" int tsdfs_set_backward_chunk(int64_t samples) {
    if (samples < 0 || samples > (int64_t)INT32_MAX / 4) return fail(TSDFS_E_INVALID, "backward chunk %lld out of range",
                                                                    (long long)samples);
    g_bwd_chunk.store(samples);
    return TSDFS_OK;
}

extern "C" int64_t tsdfs_backward_chunk_samples(const tsdfs_mlp* mlp, int64_t max_samples) {
    if (!mlp || max_samples < 1) return fail(TSDFS_E_INVALID, "mlp is NULL or max_samples < 1");
    if (mlp->arch != TSDFS_ARCH_TINY && mlp->arch != TSDFS_ARCH_ROOM) return fail(TSDFS_E_INVALID, "unknown arch %d", mlp->arch);
    return gemm_backward_chunk(mlp, max_samples);
}

extern "C" size_t tsdfs_backward_workspace_size(const tsdfs_mlp* mlp, int64_t n_rays, int64_t max_samples) {
    (void)n_rays;
    if (!mlp || max_samples < 0) return 0;
    if (mlp->arch != TSDFS_ARCH_TINY && mlp->arch != TSDFS_ARCH_ROOM) return 0;
    if (g_bwd_kind.load() == TSDFS_BACKWARD_GEMM) return gemm_backward_workspace(mlp, max_samples);
    return bwd_layout(nullptr, mlp->arch, max_samples, bwd_blocks()).bytes + 256;
}

// checks shared by the backward entry points and the training forward
static int check_mlp_and_rays(const tsdfs_mlp* mlp, const float* ray_o, const float* ray_d, const float* t_n,
                              const float* t_f, const int32_t* offsets, const uint8_t* status, int64_t n_rays,
                              int64_t max_samples) {
    if (!mlp) return fail(TSDFS_E_INVALID, "mlp is NULL");
    if (mlp->arch != TSDFS_ARCH_TINY && mlp->arch != TSDFS_ARCH_ROOM) return fail(TSDFS_E_INVALID, "unknown arch %d", mlp->arch);
    if (!mlp->sdf_w || !mlp->rgb_w) return fail(TSDFS_E_INVALID, "sdf_w and rgb_w must be non-NULL");
    if (!(mlp->scale > 0.0f) || !(mlp->beta > 0.0f) || !(mlp->inv_s > 0.0f)) return fail(TSDFS_E_INVALID, "bad mlp scalars");
    if (mlp->opacity != TSDFS_OPACITY_NEUS && mlp->opacity != TSDFS_OPACITY_VOLSDF)
        return fail(TSDFS_E_INVALID, "unknown opacity %d", mlp->opacity);
    if (n_rays < 0 || max_samples < 0) return fail(TSDFS_E_INVALID, "n_rays and max_samples must be >= 0");
    if (n_rays > 0 && (!ray_o || !ray_d || !t_n || !t_f || !offsets || !status))
        return fail(TSDFS_E_INVALID, "ray and bound pointers must be non-NULL");
    if (max_samples > (int64_t)INT32_MAX) return fail(TSDFS_E_INVALID, "max_samples must fit int32 offsets");
    return TSDFS_OK;
}

extern "C" size_t tsdfs_train_workspace_size(const tsdfs_mlp* mlp, int64_t n_rays, int64_t max_samples) {
    (void)n_rays;
    if (!mlp || max_samples < 0) return 0;
    if (mlp->arch != TSDFS_ARCH_TINY && mlp->arch != TSDFS_ARCH_ROOM) return 0;
    return gemm_backward_workspace(mlp, max_samples);
}

extern "C" int render_rays_train(const tsdfs_mlp* mlp, const float* ray_o, const float* ray_d, const float* t_n,
                                 const float* t_f, const int32_t* offsets, const uint8_t* status, int64_t n_rays,
                                 int64_t max_samples, float* rgb, float* depth, float* wsum, float* normal, float* eik,
                                 void* ws, size_t ws_bytes, tsdfs_stream_t stream) {
    int rc = check_mlp_and_rays(mlp, ray_o, ray_d, t_n, t_f, offsets, status, n_rays, max_samples);
    if (rc) return rc;
    if (n_rays == 0) return TSDFS_OK;
    if (!rgb || !depth || !wsum) return fail(TSDFS_E_INVALID, "rgb, depth and wsum must be non-NULL (normal, eik may be NULL)");
    if (!ws || ws_bytes < tsdfs_train_workspace_size(mlp, n_rays, max_samples))
        return fail(TSDFS_E_WORKSPACE, "training workspace too small");
    return gemm_train_forward(mlp, ray_o, ray_d, t_n, t_f, offsets, status, n_rays, max_samples, rgb, depth, wsum,
                              normal, eik, ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" int render_rays_backward_kept(const tsdfs_mlp* mlp, const float* ray_o, const float* ray_d,
                                         const float* t_n, const float* t_f, const int32_t* offsets,
                                         const uint8_t* status, int64_t n_rays, int64_t max_samples,
                                         const float* d_rgb, const float* d_depth, const float* d_eik,
                                         float* d_sdf_w, float* d_rgb_w, void* ws, size_t ws_bytes,
                                         tsdfs_stream_t stream) {
    int rc = check_mlp_and_rays(mlp, ray_o, ray_d, t_n, t_f, offsets, status, n_rays, max_samples);
    if (rc) return rc;
    if (n_rays == 0 || max_samples == 0) return TSDFS_OK;
    if (!d_rgb || !d_sdf_w || !d_rgb_w) return fail(TSDFS_E_INVALID, "d_rgb and gradient pointers must be non-NULL");
    if (!ws || ws_bytes < tsdfs_train_workspace_size(mlp, n_rays, max_samples))
        return fail(TSDFS_E_WORKSPACE, "training workspace too small");
    return gemm_backward(mlp, ray_o, ray_d, t_n, t_f, offsets, status, n_rays, max_samples, d_rgb, d_depth, d_eik,
                         d_sdf_w, d_rgb_w, ws, ws_bytes, (cudaStream_t)stream, true);
}

extern "C" int render_rays_backward(const tsdfs_mlp* mlp, const float* ray_o, const float* ray_d, const float* t_n,
                                    const float* t_f, const int32_t* offsets, const uint8_t* status, int64_t n_rays,
                                    int64_t max_samples, const float* d_rgb, const float* d_depth, const float* d_eik,
                                    float* d_sdf_w, float* d_rgb_w, void* ws, size_t ws_bytes, tsdfs_stream_t stream) {
    int rc = check_mlp_and_rays(mlp, ray_o, ray_d, t_n, t_f, offsets, status, n_rays, max_samples);
    if (rc) return rc;
    if (n_rays == 0) return TSDFS_OK;
    if (!d_rgb || !d_sdf_w || !d_rgb_w) return fail(TSDFS_E_INVALID, "d_rgb and gradient pointers must be non-NULL");
    if (g_bwd_kind.load() == TSDFS_BACKWARD_GEMM) {
        if (max_samples == 0) return TSDFS_OK;
        if (!ws || ws_bytes < gemm_backward_workspace(mlp, max_samples))
            return fail(TSDFS_E_WORKSPACE, "backward workspace too small");
        return gemm_backward(mlp, ray_o, ray_d, t_n, t_f, offsets, status, n_rays, max_samples, d_rgb, d_depth, d_eik,
                             d_sdf_w, d_rgb_w, ws, ws_bytes, (cudaStream_t)stream, false);
    }
    const int blocks = bwd_blocks();
    BwdWs w = bwd_layout(ws, mlp->arch, max_samples, blocks);
    if (!ws || ws_bytes < w.bytes) return fail(TSDFS_E_WORKSPACE, "backward workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    ProfScope ps("backward", st);
    NetParams np;
    np.sdf_w = mlp->sdf_w;
    np.rgb_w = mlp->rgb_w;
    for (int a = 0; a < 3; ++a) np.center[a] = mlp->center[a];
    np.scale = mlp->scale;
    np.inv_scale = 1.0f / mlp->scale;
    np.beta = mlp->beta;
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
    if (max_samples == 0) return TSDFS_OK;
    rc = mlp->arch == TSDFS_ARCH_TINY ? launch_mlp_full_simt<TSDFS_ARCH_TINY>(np, src, w.rec, max_samples, st)
                                      : launch_mlp_full_simt<TSDFS_ARCH_ROOM>(np, src, w.rec, max_samples, st);
    if (rc) return rc;
    rc = launch_comp_bwd(w.rec, offsets, status, ray_d, n_rays, mlp, d_rgb, d_depth, d_eik, w.adj, st);
    if (rc) return rc;
    const int64_t gf = mlp->arch == TSDFS_ARCH_TINY ? sdf_param_count<TSDFS_ARCH_TINY>() + rgb_param_count<TSDFS_ARCH_TINY>()
                                                    : sdf_param_count<TSDFS_ARCH_ROOM>() + rgb_param_count<TSDFS_ARCH_ROOM>();
    const int64_t n_sdf = mlp->arch == TSDFS_ARCH_TINY ? sdf_param_count<TSDFS_ARCH_TINY>() : sdf_param_count<TSDFS_ARCH_ROOM>();
    k_zero<<<grid_1d((int64_t)blocks * gf, 256), 256, 0, st>>>(w.gcopy, (int64_t)blocks * gf);
    BwdParams bp;
    bp.np = np;
    bp.src = src;
    bp.adj = w.adj;
    bp.rec = w.rec;
    bp.scratch = w.scratch;
    bp.scratch_floats = mlp->arch == TSDFS_ARCH_TINY ? scratch_floats<TSDFS_ARCH_TINY>() : scratch_floats<TSDFS_ARCH_ROOM>();
    bp.gcopy = w.gcopy;
    bp.gcopy_floats = gf;
    const size_t smem = sizeof(BwdSmem);
    static bool attr[2] = {false, false};
    if (!attr[mlp->arch]) {
        rc = cuda_check(mlp->arch == TSDFS_ARCH_TINY
                            ? cudaFuncSetAttribute(k_mlp_bwd<TSDFS_ARCH_TINY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                            : cudaFuncSetAttribute(k_mlp_bwd<TSDFS_ARCH_ROOM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                        "backward smem attribute");
        if (rc) return rc;
        attr[mlp->arch] = true;
    }
    if (mlp->arch == TSDFS_ARCH_TINY) k_mlp_bwd<TSDFS_ARCH_TINY><<<blocks, kBThreads, smem, st>>>(bp);
    else k_mlp_bwd<TSDFS_ARCH_ROOM><<<blocks, kBThreads, smem, st>>>(bp);
    rc = cuda_check(cudaGetLastError(), "backward network launch");
    if (rc) return rc;
    k_reduce_grads<<<grid_1d(gf, 256), 256, 0, st>>>(w.gcopy, blocks, gf, n_sdf, d_sdf_w, d_rgb_w);
    return cuda_check(cudaGetLastError(), "backward reduce launch");
}
