// FP64 finite-difference harness of the render's backward: the bounded render of
// render_rays (midpoint samples of [t_n, t_f], both networks with the SDF
// gradient, the network's opacity, compositing by Eq. 1 / Eq. 2) evaluated in
// FP64 on the GPU, reduced to the linear functional
//   L = sum_r g_rgb[r] . rgb[r] + g_depth[r] depth[r] + g_eik[r] eik[r]
// whose parameter gradient render_rays_backward computes.  Central differences of
// L over single parameters check that gradient.  This is test infrastructure
// (the one place the library runs FP64 arithmetic), written for clarity, not
// speed: one thread per sample walks the layers with plain loops over FP64
// weights, activations kept in a per-sample workspace slot.
#include "common.cuh"

namespace tsdfs {

namespace {

constexpr int kFdW = 320;        // widest activation row (colour input 289 <= 320)
constexpr int kFdSlot = 2 * 4 * kFdW;   // doubles per sample: two buffers of four rows

struct Fd64Net {
    const double* sdf_w;
    const double* rgb_w;
    double center[3];
    double scale, beta;
};

__device__ __forceinline__ double softplus64(double z, double beta) {
    const double bz = beta * z;
    return bz > 20.0 ? z : log1p(exp(bz)) / beta;
}
__device__ __forceinline__ double softplus_slope64(double z, double beta) {
    const double bz = beta * z;
    return bz > 20.0 ? 1.0 : 1.0 / (1.0 + exp(-bz));
}

// the positional encoding (x, sin 2^k x, cos 2^k x for k < L) of row 0 and its Jacobian
// rows 1..3 (d / dx_a), written to cols [c0, c0 + 3 + 6L) of the four rows of `h`
__device__ void encode64(const double x[3], int L, double* h, int ld, int c0, double scale_all) {
    for (int a = 0; a < 3; ++a) {
        h[c0 + a] = x[a] * scale_all;
        for (int r = 1; r < 4; ++r) h[r * ld + c0 + a] = (r - 1 == a) ? scale_all : 0.0;
    }
    for (int k = 0; k < L; ++k) {
        const double f = (double)(1 << k);
        for (int part = 0; part < 2; ++part)
            for (int a = 0; a < 3; ++a) {
                const int c = c0 + 3 + 6 * k + 3 * part + a;
                const double s = sin(f * x[a]), co = cos(f * x[a]);
                h[c] = (part == 0 ? s : co) * scale_all;
                for (int r = 1; r < 4; ++r)
                    h[r * ld + c] = (r - 1 == a) ? (part == 0 ? f * co : -f * s) * scale_all : 0.0;
            }
    }
}

template <int ARCH>
__global__ void k_fd64_samples(Fd64Net net, const float* __restrict__ ray_o, const float* __restrict__ ray_d,
                               const float* __restrict__ t_n, const float* __restrict__ t_f,
                               const int32_t* __restrict__ offsets, int64_t n_rays, int64_t total,
                               double* __restrict__ slots, double* __restrict__ rec) {
    using A = Arch<ARCH>;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int64_t r = find_ray(offsets, n_rays, g);
    const int32_t o0 = offsets[r], o1 = offsets[r + 1];
    const double tn = t_n[r], tf = t_f[r];
    const double dl = (tf - tn) / (double)(o1 - o0);
    const double t = tn + ((double)(g - o0) + 0.5) * dl;
    double o[3], d[3], xt[3];
    for (int a = 0; a < 3; ++a) {
        o[a] = ray_o[3 * r + a];
        d[a] = ray_d[3 * r + a];
        xt[a] = (o[a] + t * d[a] - net.center[a]) / net.scale;
    }
    double* buf0 = slots + g * kFdSlot;
    double* buf1 = buf0 + 4 * kFdW;
    // ---- SDF network with forward-mode tangents (rows: value, d/dx, d/dy, d/dz) ----
    encode64(xt, A::kPeSdf, buf0, kFdW, 0, 1.0);
    double* in = buf0;
    double* out = buf1;
    int width = A::kEnc;
    const double* W = net.sdf_w;
    for (int l = 0; l < A::kSdfLayers; ++l) {
        const Layer ly = A::sdf(l);
        if (l == A::kSkip) {
            // skip input concat(h, gamma(x~)) / sqrt(2)
            const double c = 1.0 / sqrt(2.0);
            for (int r = 0; r < 4; ++r)
                for (int k = 0; k < width; ++k) in[r * kFdW + k] *= c;
            encode64(xt, A::kPeSdf, in, kFdW, width, c);
            width += A::kEnc;
        }
        const double* b = W + (int64_t)ly.out * ly.in;
        const bool last = l == A::kSdfLayers - 1;
        for (int n = 0; n < ly.out; ++n) {
            double z[4] = {b[n], 0.0, 0.0, 0.0};
            for (int k = 0; k < ly.in; ++k) {
                const double w = W[(int64_t)n * ly.in + k];
                for (int rr = 0; rr < 4; ++rr) z[rr] += w * in[rr * kFdW + k];
            }
            if (last) {
                for (int rr = 0; rr < 4; ++rr) out[rr * kFdW + n] = z[rr];
            } else {
                const double sl = softplus_slope64(z[0], net.beta);
                out[n] = softplus64(z[0], net.beta);
                for (int rr = 1; rr < 4; ++rr) out[rr * kFdW + n] = sl * z[rr];
            }
        }
        W = b + ly.out;
        width = ly.out;
        double* tmp = in;
        in = out;
        out = tmp;
    }
    // in: row 0 = (net_0, feature), rows 1..3 = d net / d x~ (grad f in world units)
    const double f = net.scale * in[0];
    const double gx = in[kFdW], gy = in[2 * kFdW], gz = in[3 * kFdW];
    const double gn = sqrt(gx * gx + gy * gy + gz * gz);
    const double nh[3] = {gx / gn, gy / gn, gz / gn};
    // ---- colour network: (x~, direction encoding, unit normal, feature) ----
    const int nfeat = A::sdf(A::kSdfLayers - 1).out - 1;
    double* h = out;   // row 0 only
    for (int a = 0; a < 3; ++a) h[a] = xt[a];
    int c = 3;
    for (int a = 0; a < 3; ++a) h[c + a] = d[a];
    c += 3;
    for (int k = 0; k < A::kPeDir; ++k) {
        const double fk = (double)(1 << k);
        for (int a = 0; a < 3; ++a) h[c + a] = sin(fk * d[a]);
        for (int a = 0; a < 3; ++a) h[c + 3 + a] = cos(fk * d[a]);
        c += 6;
    }
    for (int a = 0; a < 3; ++a) h[c + a] = nh[a];
    c += 3;
    for (int j = 0; j < nfeat; ++j) h[c + j] = in[1 + j];
    double* hin = h;
    double* hout = in;
    const double* V = net.rgb_w;
    double rgb[3] = {0.0, 0.0, 0.0};
    for (int l = 0; l < A::kRgbLayers; ++l) {
        const Layer ly = A::rgb(l);
        const double* b = V + (int64_t)ly.out * ly.in;
        const bool last = l == A::kRgbLayers - 1;
        for (int n = 0; n < ly.out; ++n) {
            double z = b[n];
            for (int k = 0; k < ly.in; ++k) z += V[(int64_t)n * ly.in + k] * hin[k];
            if (last) rgb[n] = 1.0 / (1.0 + exp(-z));
            else hout[n] = z > 0.0 ? z : 0.0;
        }
        V = b + ly.out;
        double* tmp = hin;
        hin = hout;
        hout = tmp;
    }
    double* q = rec + g * 10;
    q[0] = f;
    q[1] = gx * d[0] + gy * d[1] + gz * d[2];
    q[2] = t;
    q[3] = dl;
    q[4] = rgb[0];
    q[5] = rgb[1];
    q[6] = rgb[2];
    q[7] = gn;
}

__device__ __forceinline__ double sigmoid64(double x) { return 1.0 / (1.0 + exp(-x)); }

__device__ double opacity64(int kind, double inv_s, double eps, double f, double dd, double dl) {
    if (kind == TSDFS_OPACITY_VOLSDF) {
        const double e = 0.5 * exp(-fabs(f) * inv_s);
        const double sigma = inv_s * (f >= 0.0 ? e : 1.0 - e);
        return -expm1(-sigma * dl);
    }
    const double c = dd < 0.0 ? dd : 0.0;
    const double p_lo = sigmoid64(inv_s * (f - 0.5 * dl * c));
    const double p_hi = sigmoid64(inv_s * (f + 0.5 * dl * c));
    double a = (p_lo - p_hi + eps) / (p_lo + eps);
    return a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
}

__global__ void k_fd64_rays(const double* __restrict__ rec, const int32_t* __restrict__ offsets,
                            const uint8_t* __restrict__ status, int64_t n_rays, int kind, double inv_s, double eps,
                            const float* __restrict__ g_rgb, const float* __restrict__ g_depth,
                            const float* __restrict__ g_eik, double* __restrict__ contrib) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const int64_t b = offsets[r];
    const int64_t e = status[r] == TSDFS_MISS ? b : offsets[r + 1];
    double logT = 0.0, ws = 0.0, c[3] = {0.0, 0.0, 0.0}, dt = 0.0, eik = 0.0;
    const double clamp = 1.0 - 5.9604644775390625e-8;   // 1 - 2^-24
    for (int64_t g = b; g < e; ++g) {
        const double* q = rec + g * 10;
        const double alpha = opacity64(kind, inv_s, eps, q[0], q[1], q[3]);
        const double w = exp(logT) * alpha;
        ws += w;
        for (int a = 0; a < 3; ++a) c[a] += w * q[4 + a];
        dt += w * q[2];
        eik += (q[7] - 1.0) * (q[7] - 1.0);
        logT += log1p(-(alpha < clamp ? alpha : clamp));
    }
    const double depth = ws >= 1e-8 ? dt / ws : 0.0;
    double v = 0.0;
    for (int a = 0; a < 3; ++a) v += (double)g_rgb[3 * r + a] * c[a];
    if (g_depth) v += (double)g_depth[r] * depth;
    if (g_eik && status[r] == TSDFS_BOUNDED) v += (double)g_eik[r] * eik;
    contrib[r] = v;
}

// one block: the rays' contributions summed in a fixed order
__global__ void k_fd64_sum(const double* __restrict__ contrib, int64_t n_rays, double* __restrict__ loss) {
    __shared__ double part[256];
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < n_rays; r += blockDim.x) s += contrib[r];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = part[0];
}

int64_t fd64_ws(int64_t n_rays, int64_t max_samples) {
    return (int64_t)sizeof(double) * (max_samples * (int64_t)(kFdSlot + 10) + n_rays) + 256;
}

}  // namespace

}  // namespace tsdfs

using namespace tsdfs;

extern "C" size_t tsdfs_loss_f64_workspace_size(int64_t n_rays, int64_t max_samples) {
    if (n_rays < 0 || max_samples < 0) return 0;
    return (size_t)fd64_ws(n_rays, max_samples);
}

extern "C" int tsdfs_loss_f64(const tsdfs_mlp* m, const double* sdf_w64, const double* rgb_w64, const float* ray_o,
                              const float* ray_d, const float* t_n, const float* t_f, const int32_t* offsets,
                              const uint8_t* status, int64_t n_rays, int64_t max_samples, const float* g_rgb,
                              const float* g_depth, const float* g_eik, double* loss, void* ws, size_t ws_bytes,
                              tsdfs_stream_t stream) {
    if (!m || (m->arch != TSDFS_ARCH_TINY && m->arch != TSDFS_ARCH_ROOM))
        return fail(TSDFS_E_INVALID, "tsdfs_loss_f64: unknown network");
    if (!sdf_w64 || !rgb_w64 || !ray_o || !ray_d || !t_n || !t_f || !offsets || !status || !g_rgb || !loss || !ws)
        return fail(TSDFS_E_INVALID, "tsdfs_loss_f64: a required pointer is NULL");
    if (n_rays < 1 || max_samples < 1) return fail(TSDFS_E_INVALID, "tsdfs_loss_f64: n_rays and max_samples must be >= 1");
    if (ws_bytes < (size_t)fd64_ws(n_rays, max_samples))
        return fail(TSDFS_E_WORKSPACE, "tsdfs_loss_f64: workspace too small");
    if (m->opacity != TSDFS_OPACITY_NEUS && m->opacity != TSDFS_OPACITY_VOLSDF)
        return fail(TSDFS_E_INVALID, "tsdfs_loss_f64: unknown opacity");
    cudaStream_t st = (cudaStream_t)stream;
    // the sample total is read once on the host (test infrastructure: synchronising is fine)
    int32_t total = 0;
    int rc = cuda_check(cudaMemcpyAsync(&total, offsets + n_rays, sizeof(total), cudaMemcpyDeviceToHost, st),
                        "tsdfs_loss_f64 total");
    if (rc) return rc;
    rc = cuda_check(cudaStreamSynchronize(st), "tsdfs_loss_f64 synchronize");
    if (rc) return rc;
    if (total < 0 || total > max_samples) return fail(TSDFS_E_WORKSPACE, "tsdfs_loss_f64: %d samples > max_samples", total);
    double* base = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255));
    double* slots = base;
    double* rec = slots + max_samples * (int64_t)kFdSlot;
    double* contrib = rec + max_samples * 10;
    Fd64Net net{sdf_w64, rgb_w64, {m->center[0], m->center[1], m->center[2]}, (double)m->scale, (double)m->beta};
    if (total > 0) {
        const int blk = 32;   // spread the few samples over many SMs
        const unsigned grid = (unsigned)((total + blk - 1) / blk);
        if (m->arch == TSDFS_ARCH_TINY)
            k_fd64_samples<TSDFS_ARCH_TINY><<<grid, blk, 0, st>>>(net, ray_o, ray_d, t_n, t_f, offsets, n_rays, total,
                                                                  slots, rec);
        else
            k_fd64_samples<TSDFS_ARCH_ROOM><<<grid, blk, 0, st>>>(net, ray_o, ray_d, t_n, t_f, offsets, n_rays, total,
                                                                  slots, rec);
        rc = cuda_check(cudaGetLastError(), "tsdfs_loss_f64 samples launch");
        if (rc) return rc;
    }
    k_fd64_rays<<<(unsigned)((n_rays + 127) / 128), 128, 0, st>>>(rec, offsets, status, n_rays, m->opacity,
                                                                 (double)m->inv_s, (double)m->alpha_eps, g_rgb, g_depth,
                                                                 g_eik, contrib);
    rc = cuda_check(cudaGetLastError(), "tsdfs_loss_f64 rays launch");
    if (rc) return rc;
    k_fd64_sum<<<1, 256, 0, st>>>(contrib, n_rays, loss);
    return cuda_check(cudaGetLastError(), "tsdfs_loss_f64 sum launch");
}
