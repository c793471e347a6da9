// Layer-major backward of render_rays on the tensor cores.
//
// Each layer of both networks is a GEMM over a chunk of n samples.  The SDF
// network's rows are the value row and the three forward-mode tangent rows of
// every sample (4n rows; the bias enters the value rows only); the colour
// network has one row per sample.  With X_l a layer's input rows, P_l = X_l W_l^T
// its pre-activation without the bias, and G_l the adjoint of P_l:
//   forward   P_l = X_l W_l^T
//   backward  dW_l += G_l^T X_l,  db_l += sum of G_l over the bias rows,  D_l = G_l W_l
// (D_l: the adjoint of X_l).  The element-wise steps between the GEMMs are the
// kernels of this file: the SDF input encoding and its x-derivatives; softplus
// on value rows and the slope sigma(beta z) times the tangent rows; the skip
// concatenation; the SDF output (f, grad f, the unit normal, the colour input);
// ReLU and sigmoid.  Backwards: the sigmoid and ReLU masks, the adjoint of the
// SDF output (f, grad f through the unit normal, and the colour input's feature
// columns), and the softplus layer's adjoint including its second-order term
// (the tangent rows' slope depends on z: d sigma / dz = beta sigma (1 - sigma)).
//
// The GEMMs run in cuBLAS with FP32 operands emulated on the BF16 tensor cores
// (each operand split into three BF16 parts, FP32 accumulation:
// CUBLAS_COMPUTE_32F_EMULATED_16BFX9), without the emulation's handling of
// infinite and NaN operands: the parameters are checked for non-finite values
// (TSDFS_DEV_NONFINITE) instead.  Every matrix is row-major with both of its
// widths padded to a multiple of 4 floats (16 bytes), zero in the padding, which
// keeps every GEMM on the tensor-core kernels; the weights are copied once per
// call into that padded layout, and the gradients accumulate in a padded scratch
// that is added into the caller's packed gradients at the end.
//
// The sample total sizes the GEMMs, so the call reads it from the device first
// (one synchronisation of the stream).  When all samples fit one chunk, the
// forward pass that makes the per-sample records keeps its activations for the
// backward; otherwise pass 1 makes the records chunk by chunk, the compositing
// backward runs over all rays, and pass 2 recomputes each chunk's activations
// before back-propagating through it.
#include <cublas_v2.h>

#include <mutex>

#include "backward.cuh"

namespace tsdfs {
int launch_composite(const SampleRec* rec, const int32_t* offsets, int per_ray, const uint8_t* status, int64_t n_rays,
                     const int32_t* total_dev, int64_t capacity, Opacity op, float* rgb, float* depth,
                     float* wsum, float* normal, float* eik, cudaStream_t st);
}  // namespace tsdfs

namespace tsdfs {
namespace {

constexpr int64_t kDefaultChunkBytes = 16ll << 30;  // activations of one chunk
constexpr size_t kBlasWorkspace = 64u << 20;        // cuBLAS workspace inside the caller's
constexpr int kEw = 256;                            // threads of the element-wise kernels
constexpr float kSkipScale = 0.70710678118654752f;  // 1 / sqrt(2) at the skip concatenation

__host__ __device__ constexpr int pad4(int n) { return (n + 3) & ~3; }

// padded layout of one architecture: weights W [pad4(out)][pad4(in)] then b [pad4(out)]
// per layer, the SDF layers first; activation rows padded to pad4(width)
template <int ARCH>
struct GLayout {
    using A = Arch<ARCH>;
    static constexpr int LS = A::kSdfLayers, LC = A::kRgbLayers;
    __host__ __device__ static constexpr int64_t layer_floats(Layer ly) {
        return (int64_t)pad4(ly.out) * pad4(ly.in) + pad4(ly.out);
    }
    __host__ __device__ static constexpr int64_t sdf_off(int l) {
        int64_t o = 0;
        for (int i = 0; i < l; ++i) o += layer_floats(A::sdf(i));
        return o;
    }
    __host__ __device__ static constexpr int64_t rgb_off(int l) {
        int64_t o = sdf_off(LS);
        for (int i = 0; i < l; ++i) o += layer_floats(A::rgb(i));
        return o;
    }
    __host__ __device__ static constexpr int64_t total() { return rgb_off(LC); }
    // widest SDF row (inputs and outputs), the row length of the G / D work buffers
    static constexpr int max_sdf_width() {
        int w = 0;
        for (int l = 0; l < LS; ++l) {
            w = pad4(A::sdf(l).in) > w ? pad4(A::sdf(l).in) : w;
            w = pad4(A::sdf(l).out) > w ? pad4(A::sdf(l).out) : w;
        }
        return w;
    }
    static constexpr int max_rgb_width() {
        int w = 0;
        for (int l = 0; l < LC; ++l) {
            w = pad4(A::rgb(l).in) > w ? pad4(A::rgb(l).in) : w;
            w = pad4(A::rgb(l).out) > w ? pad4(A::rgb(l).out) : w;
        }
        return w;
    }
    // floats of one work buffer per sample: 4 SDF rows or one colour row, whichever is wider
    static constexpr int64_t work_floats() {
        return 4 * max_sdf_width() > max_rgb_width() ? 4 * max_sdf_width() : max_rgb_width();
    }
    // floats of activations kept per sample (X_l and P_l of every layer)
    static constexpr int64_t act_floats() {
        int64_t n = 0;
        for (int l = 0; l < LS; ++l) n += 4 * (int64_t)(pad4(A::sdf(l).in) + pad4(A::sdf(l).out));
        for (int l = 0; l < LC; ++l) n += (int64_t)pad4(A::rgb(l).in) + pad4(A::rgb(l).out);
        return n;
    }
};

struct __align__(16) SampleAux {
    float xt[3];   // normalised position x~ = (o + t d - c) / scale
    float t;       // sample position along the ray
    float dir[3];  // ray direction
    float dl;      // section width
};

// ---- weight and gradient layouts ------------------------------------------------

// copy the packed parameters into the padded layout (zero padding)
template <int ARCH>
__global__ void k_pad_weights(const float* __restrict__ sdf_w, const float* __restrict__ rgb_w, float* __restrict__ wp) {
    using A = Arch<ARCH>;
    using L = GLayout<ARCH>;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L::total(); i += (int64_t)gridDim.x * blockDim.x) {
        const bool sdf = i < L::sdf_off(L::LS);
        const int nl = sdf ? L::LS : L::LC;
        int l = 0;
        while (l + 1 < nl && i >= (sdf ? L::sdf_off(l + 1) : L::rgb_off(l + 1))) ++l;
        const Layer ly = sdf ? A::sdf(l) : A::rgb(l);
        const int64_t e = i - (sdf ? L::sdf_off(l) : L::rgb_off(l));
        const float* src = sdf ? sdf_w + sdf_layer_offset<ARCH>(l) : rgb_w + rgb_layer_offset<ARCH>(l);
        const int kp = pad4(ly.in);
        float v = 0.0f;
        if (e < (int64_t)pad4(ly.out) * kp) {
            const int n = (int)(e / kp), k = (int)(e % kp);
            if (n < ly.out && k < ly.in) v = src[(int64_t)n * ly.in + k];
        } else {
            const int n = (int)(e - (int64_t)pad4(ly.out) * kp);
            if (n < ly.out) v = src[(int64_t)ly.out * ly.in + n];
        }
        wp[i] = v;
    }
}

// d_sdf_w / d_rgb_w (packed layout) += the padded gradient scratch
template <int ARCH>
__global__ void k_add_grads(const float* __restrict__ dwp, float* __restrict__ d_sdf, float* __restrict__ d_rgb) {
    using A = Arch<ARCH>;
    using L = GLayout<ARCH>;
    constexpr int64_t n_sdf = sdf_param_count<ARCH>(), n_all = n_sdf + rgb_param_count<ARCH>();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_all; i += (int64_t)gridDim.x * blockDim.x) {
        const bool sdf = i < n_sdf;
        const int64_t j = sdf ? i : i - n_sdf;
        const int nl = sdf ? L::LS : L::LC;
        int l = 0;
        while (l + 1 < nl && j >= (sdf ? sdf_layer_offset<ARCH>(l + 1) : rgb_layer_offset<ARCH>(l + 1))) ++l;
        const Layer ly = sdf ? A::sdf(l) : A::rgb(l);
        const int64_t e = j - (sdf ? sdf_layer_offset<ARCH>(l) : rgb_layer_offset<ARCH>(l));
        const int64_t po = sdf ? L::sdf_off(l) : L::rgb_off(l);
        const int kp = pad4(ly.in);
        float v;
        if (e < (int64_t)ly.out * ly.in) v = dwp[po + (e / ly.in) * kp + e % ly.in];
        else v = dwp[po + (int64_t)pad4(ly.out) * kp + (e - (int64_t)ly.out * ly.in)];
        if (sdf) d_sdf[j] += v;
        else d_rgb[j] += v;
    }
}

__global__ void k_fill(float* __restrict__ p, int64_t n, float v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

__global__ void k_flag_overflow(const int32_t* __restrict__ total, int64_t capacity, uint32_t* status) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && (int64_t)*total > capacity) set_status(status, TSDFS_DEV_SAMPLES_OVERFLOW);
}

// TSDFS_DEV_NONFINITE when a parameter is infinite or NaN (the GEMMs assume finite operands)
__global__ void k_check_params(const float* __restrict__ sdf_w, int64_t n_sdf, const float* __restrict__ rgb_w,
                               int64_t n_rgb, uint32_t* status) {
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_sdf + n_rgb; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = i < n_sdf ? sdf_w[i] : rgb_w[i - n_sdf];
        bad = bad || !isfinite(v);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) set_status(status, TSDFS_DEV_NONFINITE);
}

// ---- forward element-wise steps -------------------------------------------------

// sample positions of samples c0 .. c0 + n - 1 (midpoints of [t_n, t_f], ragged offsets)
__global__ void k_gsetup(NetParams np, SampleSource src, int64_t c0, int64_t n, SampleAux* __restrict__ aux) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = c0 + s;
        const int64_t r = find_ray(src.offsets, src.n_rays, g);
        const int i = (int)(g - __ldg(src.offsets + r));
        const int cnt = __ldg(src.offsets + r + 1) - __ldg(src.offsets + r);
        const float tn = __ldg(src.t_n + r), tf = __ldg(src.t_f + r);
        const float dl = (tf - tn) / (float)cnt;
        const float t = tn + ((float)i + 0.5f) * dl;
        SampleAux a;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float o = __ldg(src.ray_o + 3 * r + k), d = __ldg(src.ray_d + 3 * r + k);
            a.xt[k] = (o + t * d - np.center[k]) * np.inv_scale;
            a.dir[k] = d;
        }
        a.t = t;
        a.dl = dl;
        aux[s] = a;
    }
}

// SDF input rows: row 4s = gamma(x~), rows 4s + 1 + a = d gamma / d x~_a (Sec. 3.1
// positional encoding: x~, then per octave k sin(2^k x~), cos(2^k x~))
template <int ARCH>
__global__ void k_genc(const SampleAux* __restrict__ aux, int64_t n, float* __restrict__ X0) {
    using A = Arch<ARCH>;
    constexpr int E = A::kEnc, ld = pad4(E);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * ld; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = e / ld;
        const int k = (int)(e % ld);
        float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (k < 3) {
            v[0] = aux[s].xt[k];
            v[1 + k] = 1.0f;
        } else if (k < E) {
            const int q = k - 3, oct = q / 6, part = (q % 6) / 3, b = q % 3;
            const float f = (float)(1 << oct);
            float sn, cs;
            sincosf(f * aux[s].xt[b], &sn, &cs);
            v[0] = part == 0 ? sn : cs;
            v[1 + b] = part == 0 ? f * cs : -f * sn;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) X0[(4 * s + c) * ld + k] = v[c];
    }
}

// next SDF layer input from P (hidden layer of width No): value rows softplus_beta(z),
// tangent rows sigma(beta z) dz; scaled by sc, with the encoding rows appended at
// the skip input
__global__ void k_gsp_fwd(const float* __restrict__ P, int ldp, const float* __restrict__ bias, int No,
                          const float* __restrict__ X0, int ldx0, int E, bool skip, float sc, float beta, int64_t n,
                          float* __restrict__ Xn, int ldxn) {
    // one thread per sample and group of 4 columns (every row length is a multiple of 4, so
    // the P, bias and Xn accesses are 16-byte vectors; P and bias hold pad4(No) columns)
    const int q4 = ldxn / 4;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * q4; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = e / q4;
        const int j0 = 4 * (int)(e % q4);
        float v[4][4] = {};   // [row][column]
        float pz[4] = {}, pt[3][4] = {}, bz4[4] = {};
        if (j0 < No) {
            const float4 z = *reinterpret_cast<const float4*>(P + 4 * s * ldp + j0);
            const float4 b = __ldg(reinterpret_cast<const float4*>(bias + j0));
            pz[0] = z.x; pz[1] = z.y; pz[2] = z.z; pz[3] = z.w;
            bz4[0] = b.x; bz4[1] = b.y; bz4[2] = b.z; bz4[3] = b.w;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float4 t = *reinterpret_cast<const float4*>(P + (4 * s + 1 + a) * ldp + j0);
                pt[a][0] = t.x; pt[a][1] = t.y; pt[a][2] = t.z; pt[a][3] = t.w;
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int j = j0 + i;
            if (j < No) {
                const float zz = pz[i] + bz4[i];
                const float bz = beta * zz;
                const float sg = bz > 20.0f ? 1.0f : 1.0f / (1.0f + expf(-bz));
                v[0][i] = sc * (bz > 20.0f ? zz : log1pf(expf(bz)) / beta);
#pragma unroll
                for (int a = 1; a < 4; ++a) v[a][i] = sc * sg * pt[a - 1][i];
            } else if (skip && j < No + E) {
#pragma unroll
                for (int c = 0; c < 4; ++c) v[c][i] = sc * X0[(4 * s + c) * ldx0 + (j - No)];
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
            *reinterpret_cast<float4*>(Xn + (4 * s + c) * ldxn + j0) = make_float4(v[c][0], v[c][1], v[c][2], v[c][3]);
    }
}

// SDF output [net_0, feature] -> the record's f, grad f, unit normal, and the colour
// input row [x~, direction encoding, unit normal, feature]
template <int ARCH>
__global__ void k_gsdf_out(const float* __restrict__ P, int ldp, const float* __restrict__ bias,
                           const SampleAux* __restrict__ aux, int64_t n, int64_t c0, float scale,
                           float* __restrict__ Xc, int ldxc, SampleRec* __restrict__ rec) {
    using A = Arch<ARCH>;
    constexpr int kDir = A::kDirEnc, fo = 3 + kDir + 3, Kc = A::rgb(0).in;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * ldxc; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = e / ldxc;
        const int j = (int)(e % ldxc);
        const SampleAux& a = aux[s];
        const float* Pv = P + 4 * s * ldp;
        float v = 0.0f;
        const bool need_g = j == 0 || (j >= 3 + kDir && j < fo);
        float gx = 0.0f, gy = 0.0f, gz = 0.0f, gn = 0.0f, inv = 0.0f;
        if (need_g) {
            gx = Pv[ldp];
            gy = Pv[2 * ldp];
            gz = Pv[3 * ldp];
            gn = sqrtf(gx * gx + gy * gy + gz * gz);
            inv = gn > 0.0f ? 1.0f / gn : 0.0f;
        }
        if (j < 3) {
            v = a.xt[j];
        } else if (j < 3 + kDir) {
            const int q = j - 3;
            if (q < 3) {
                v = a.dir[q];
            } else {
                const int q2 = q - 3, oct = q2 / 6, part = (q2 % 6) / 3, b = q2 % 3;
                float sn, cs;
                sincosf((float)(1 << oct) * a.dir[b], &sn, &cs);
                v = part == 0 ? sn : cs;
            }
        } else if (j < fo) {
            const int c = j - 3 - kDir;
            v = (c == 0 ? gx : (c == 1 ? gy : gz)) * inv;
        } else if (j < Kc) {
            v = Pv[1 + j - fo] + __ldg(bias + 1 + j - fo);
        }
        Xc[s * ldxc + j] = v;
        if (j == 0) {
            SampleRec& R = rec[c0 + s];
            R.f = scale * (Pv[0] + __ldg(bias));
            R.dd = gx * a.dir[0] + gy * a.dir[1] + gz * a.dir[2];
            R.t = a.t;
            R.delta = a.dl;
            R.gnorm = gn;
            R.nx = gx * inv;
            R.ny = gy * inv;
            R.nz = gz * inv;
            R.pad = 0.0f;
        }
    }
}

// next colour layer input: ReLU(P + b), zero padding
__global__ void k_grelu_fwd(const float* __restrict__ P, int ldp, const float* __restrict__ bias, int N, int64_t n,
                            float* __restrict__ Xn, int ldxn) {
    // 4 columns per thread as 16-byte vectors (P and bias hold pad4(N) columns, ldxn too)
    const int q4 = ldxn / 4;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * q4; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = e / q4;
        const int j0 = 4 * (int)(e % q4);
        float4 o = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (j0 < N) {
            const float4 pv = *reinterpret_cast<const float4*>(P + s * ldp + j0);
            const float4 bv = __ldg(reinterpret_cast<const float4*>(bias + j0));
            o.x = fmaxf(pv.x + bv.x, 0.0f);
            o.y = j0 + 1 < N ? fmaxf(pv.y + bv.y, 0.0f) : 0.0f;
            o.z = j0 + 2 < N ? fmaxf(pv.z + bv.z, 0.0f) : 0.0f;
            o.w = j0 + 3 < N ? fmaxf(pv.w + bv.w, 0.0f) : 0.0f;
        }
        *reinterpret_cast<float4*>(Xn + s * ldxn + j0) = o;
    }
}

// colour = sigmoid(P + b) into the records
__global__ void k_grgb_out(const float* __restrict__ P, int ldp, const float* __restrict__ bias, int64_t n, int64_t c0,
                           SampleRec* __restrict__ rec) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        SampleRec& R = rec[c0 + s];
        R.r = 1.0f / (1.0f + expf(-(P[s * ldp + 0] + __ldg(bias + 0))));
        R.g = 1.0f / (1.0f + expf(-(P[s * ldp + 1] + __ldg(bias + 1))));
        R.b = 1.0f / (1.0f + expf(-(P[s * ldp + 2] + __ldg(bias + 2))));
    }
}

// ---- backward element-wise steps ------------------------------------------------

// adjoint of the colour output layer's pre-activation: d rgb * y (1 - y)
__global__ void k_grgb_bwd(const float* __restrict__ P, int ldp, const float* __restrict__ bias,
                           const SampleAdj* __restrict__ adj, int64_t n, int64_t c0, float* __restrict__ G, int ldg) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const SampleAdj& A = adj[c0 + s];
        const float gy[3] = {A.gr, A.gg, A.gb};
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float y = 1.0f / (1.0f + expf(-(P[s * ldp + ch] + __ldg(bias + ch))));
            G[s * ldg + ch] = gy[ch] * y * (1.0f - y);
        }
        for (int ch = 3; ch < ldg; ++ch) G[s * ldg + ch] = 0.0f;
    }
}

// through a hidden colour layer's ReLU: G = D where P + b > 0 (zero padding)
__global__ void k_grelu_bwd(const float* __restrict__ D, int ldd, const float* __restrict__ P, int ldp,
                            const float* __restrict__ bias, int N, int64_t n, float* __restrict__ G, int ldg) {
    // 4 columns per thread as 16-byte vectors (D, P and bias hold at least pad4(N) columns)
    const int q4 = ldg / 4;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * q4; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = e / q4;
        const int j0 = 4 * (int)(e % q4);
        float4 o = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (j0 < N) {
            const float4 dv = *reinterpret_cast<const float4*>(D + s * ldd + j0);
            const float4 pv = *reinterpret_cast<const float4*>(P + s * ldp + j0);
            const float4 bv = __ldg(reinterpret_cast<const float4*>(bias + j0));
            o.x = pv.x + bv.x > 0.0f ? dv.x : 0.0f;
            o.y = j0 + 1 < N && pv.y + bv.y > 0.0f ? dv.y : 0.0f;
            o.z = j0 + 2 < N && pv.z + bv.z > 0.0f ? dv.z : 0.0f;
            o.w = j0 + 3 < N && pv.w + bv.w > 0.0f ? dv.w : 0.0f;
        }
        *reinterpret_cast<float4*>(G + s * ldg + j0) = o;
    }
}

// adjoint of the SDF output rows from the per-sample adjoints and the colour input's:
// value row [scale * d f, d feature]; tangent row a [d (grad f)_a + the unit normal's
// share (d n^_a - n^_a (n^ . d n^)) / |grad f|, 0 ...]
template <int ARCH>
__global__ void k_gsdf_out_bwd(const float* __restrict__ D, int ldd, const SampleAdj* __restrict__ adj,
                               const SampleRec* __restrict__ rec, int64_t n, int64_t c0, float scale,
                               float* __restrict__ G, int ldg) {
    using A = Arch<ARCH>;
    constexpr int kDir = A::kDirEnc, fo = 3 + kDir + 3, No = A::sdf(A::kSdfLayers - 1).out;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * ldg; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = e / ldg;
        const int j = (int)(e % ldg);
        float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (j >= No) {
            // padding
        } else if (j == 0) {
            const SampleAdj& Ad = adj[c0 + s];
            const SampleRec& R = rec[c0 + s];
            v[0] = Ad.gf * scale;
            const float nh[3] = {R.nx, R.ny, R.nz};
            const float* dn = D + s * ldd + 3 + kDir;
            const float dot = nh[0] * dn[0] + nh[1] * dn[1] + nh[2] * dn[2];
            const float gg[3] = {Ad.ggx, Ad.ggy, Ad.ggz};
#pragma unroll
            for (int c = 0; c < 3; ++c) v[1 + c] = gg[c] + (R.gnorm > 0.0f ? (dn[c] - nh[c] * dot) / R.gnorm : 0.0f);
        } else {
            v[0] = D[s * ldd + fo + j - 1];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) G[(4 * s + c) * ldg + j] = v[c];
    }
}

// adjoint of a hidden SDF layer's pre-activation rows from the adjoint D of the next
// layer's input (its first N columns; the encoding columns of the skip input carry no
// parameter gradient): tangent rows sc sigma D_a, value row
// sc (sigma D_0 + sigma' sum_a D_a dz_a)
__global__ void k_gsp_bwd(const float* __restrict__ D, int ldd, const float* __restrict__ P, int ldp,
                          const float* __restrict__ bias, int N, float sc, float beta, int64_t n,
                          float* __restrict__ G, int ldg) {
    // one thread per sample and group of 4 columns (16-byte vectors: every row length is a
    // multiple of 4, and D, P and bias hold at least pad4(N) columns)
    const int q4 = ldg / 4;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * q4; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = e / q4;
        const int j0 = 4 * (int)(e % q4);
        float g[4][4] = {};   // [row][column]
        if (j0 < N) {
            float d[4][4], p[4][4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float4 dv = *reinterpret_cast<const float4*>(D + (4 * s + r) * ldd + j0);
                const float4 pv = *reinterpret_cast<const float4*>(P + (4 * s + r) * ldp + j0);
                d[r][0] = dv.x; d[r][1] = dv.y; d[r][2] = dv.z; d[r][3] = dv.w;
                p[r][0] = pv.x; p[r][1] = pv.y; p[r][2] = pv.z; p[r][3] = pv.w;
            }
            const float4 bv = __ldg(reinterpret_cast<const float4*>(bias + j0));
            b[0] = bv.x; b[1] = bv.y; b[2] = bv.z; b[3] = bv.w;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (j0 + i >= N) continue;
                const float bz = beta * (p[0][i] + b[i]);
                const float sg = bz > 20.0f ? 1.0f : 1.0f / (1.0f + expf(-bz));
                const float dsg = bz > 20.0f ? 0.0f : beta * sg * (1.0f - sg);
                float second = 0.0f;
#pragma unroll
                for (int a = 1; a < 4; ++a) second += d[a][i] * p[a][i];
                g[0][i] = sc * (sg * d[0][i] + dsg * second);
#pragma unroll
                for (int a = 1; a < 4; ++a) g[a][i] = sc * sg * d[a][i];
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
            *reinterpret_cast<float4*>(G + (4 * s + r) * ldg + j0) = make_float4(g[r][0], g[r][1], g[r][2], g[r][3]);
    }
}

// ---- cuBLAS -------------------------------------------------------------------------

struct BlasCache {
    std::mutex mu;
    cublasHandle_t h[SymbolCache::kDevices] = {};
    unsigned long long ctx[SymbolCache::kDevices] = {};
};
BlasCache g_blas;

int blas_check(cublasStatus_t s, const char* what) {
    if (s == CUBLAS_STATUS_SUCCESS) return TSDFS_OK;
    return fail(TSDFS_E_CUDA, "cuBLAS %s: status %d", what, (int)s);
}

// the device's handle, made again when the device's context has changed (after a
// cudaDeviceReset); called with g_blas.mu held
int blas_handle(cublasHandle_t* out) {
    int dev = 0;
    int rc = cuda_check(cudaGetDevice(&dev), "backward device");
    if (rc) return rc;
    if (dev < 0 || dev >= SymbolCache::kDevices) return fail(TSDFS_E_UNSUPPORTED, "device index %d out of range", dev);
    const unsigned long long id = current_context_id();
    if (g_blas.h[dev] && id != 0 && id == g_blas.ctx[dev]) {
        *out = g_blas.h[dev];
        return TSDFS_OK;
    }
    cublasHandle_t h = nullptr;
    rc = blas_check(cublasCreate(&h), "create");
    if (rc) return rc;
    rc = blas_check(cublasSetPointerMode(h, CUBLAS_POINTER_MODE_HOST), "pointer mode");
    if (!rc) rc = blas_check(cublasSetEmulationSpecialValuesSupport(h, CUDA_EMULATION_SPECIAL_VALUES_SUPPORT_NONE),
                             "emulation special values");
    if (rc) return rc;
    g_blas.h[dev] = h;
    g_blas.ctx[dev] = id ? id : current_context_id();
    *out = h;
    return TSDFS_OK;
}

// Row-major products in cuBLAS's column-major terms (a row-major M x K matrix with row
// length ld is a column-major K x M matrix with leading dimension ld):
// P [R x N] = X [R x K] W^T, W [N x K]
int mm_fwd(cublasHandle_t h, int64_t R, int K, int N, const float* X, int ldx, const float* W, int ldw, float* P, int ldp) {
    const float one = 1.0f, zero = 0.0f;
    return blas_check(cublasGemmEx(h, CUBLAS_OP_T, CUBLAS_OP_N, N, (int)R, K, &one, W, CUDA_R_32F, ldw, X, CUDA_R_32F, ldx,
                                   &zero, P, CUDA_R_32F, ldp, CUBLAS_COMPUTE_32F_EMULATED_16BFX9, CUBLAS_GEMM_DEFAULT),
                      "forward GEMM");
}

// D [R x K] = G [R x N] W, W [N x K]
int mm_dx(cublasHandle_t h, int64_t R, int N, int K, const float* G, int ldg, const float* W, int ldw, float* D, int ldd) {
    const float one = 1.0f, zero = 0.0f;
    return blas_check(cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, K, (int)R, N, &one, W, CUDA_R_32F, ldw, G, CUDA_R_32F, ldg,
                                   &zero, D, CUDA_R_32F, ldd, CUBLAS_COMPUTE_32F_EMULATED_16BFX9, CUBLAS_GEMM_DEFAULT),
                      "input-adjoint GEMM");
}

// dW [N x K] += G^T X, G [R x N], X [R x K]
int mm_dw(cublasHandle_t h, int64_t R, int N, int K, const float* G, int ldg, const float* X, int ldx, float* dW, int lddw) {
    const float one = 1.0f;
    return blas_check(cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_T, K, N, (int)R, &one, X, CUDA_R_32F, ldx, G, CUDA_R_32F, ldg,
                                   &one, dW, CUDA_R_32F, lddw, CUBLAS_COMPUTE_32F_EMULATED_16BFX9, CUBLAS_GEMM_DEFAULT),
                      "weight-gradient GEMM");
}

// db [N] += sum over n rows of G taken every `stride` rows (stride 4: the SDF value rows)
int mv_db(cublasHandle_t h, int64_t n, int N, const float* G, int ldg, int stride, const float* ones, float* db) {
    const float one = 1.0f;
    return blas_check(cublasSgemv(h, CUBLAS_OP_N, N, (int)n, &one, G, ldg * stride, ones, 1, &one, db, 1), "bias-gradient GEMV");
}

// ---- workspace ----------------------------------------------------------------------

template <int ARCH>
struct GemmWs {
    using L = GLayout<ARCH>;
    SampleRec* rec;
    SampleAdj* adj;
    float* wp;     // padded weights
    float* dwp;    // padded gradients
    void* blas;
    float* ones;
    SampleAux* aux;
    float* G;
    float* D;
    float* X[L::LS];
    float* P[L::LS];
    float* Xc[L::LC];
    float* Pc[L::LC];
    int64_t chunk;  // samples per chunk
    size_t bytes;
};

template <int ARCH>
int64_t chunk_samples(int64_t max_samples) {
    using L = GLayout<ARCH>;
    const int64_t per = (L::act_floats() + 2 * L::work_floats() + 1) * 4 + (int64_t)sizeof(SampleAux);
    int64_t c = backward_chunk_setting();
    if (c <= 0) c = kDefaultChunkBytes / per;
    if (c > max_samples) c = max_samples;
    return c < 1 ? 1 : c;
}

template <int ARCH>
GemmWs<ARCH> gemm_layout(void* base, int64_t max_samples) {
    using A = Arch<ARCH>;
    using L = GLayout<ARCH>;
    GemmWs<ARCH> w{};
    uintptr_t p = (reinterpret_cast<uintptr_t>(base) + 255) & ~uintptr_t(255);
    const uintptr_t p0 = p;
    auto take = [&](size_t bytes) {
        uintptr_t q = p;
        p = (p + bytes + 255) & ~uintptr_t(255);
        return q;
    };
    const int64_t C = chunk_samples<ARCH>(max_samples);
    w.chunk = C;
    w.rec = reinterpret_cast<SampleRec*>(take((size_t)max_samples * sizeof(SampleRec)));
    w.adj = reinterpret_cast<SampleAdj*>(take((size_t)max_samples * sizeof(SampleAdj)));
    w.wp = reinterpret_cast<float*>(take((size_t)L::total() * 4));
    w.dwp = reinterpret_cast<float*>(take((size_t)L::total() * 4));
    w.blas = reinterpret_cast<void*>(take(kBlasWorkspace));
    w.ones = reinterpret_cast<float*>(take((size_t)C * 4));
    w.aux = reinterpret_cast<SampleAux*>(take((size_t)C * sizeof(SampleAux)));
    w.G = reinterpret_cast<float*>(take((size_t)C * L::work_floats() * 4));
    w.D = reinterpret_cast<float*>(take((size_t)C * L::work_floats() * 4));
    for (int l = 0; l < L::LS; ++l) {
        w.X[l] = reinterpret_cast<float*>(take((size_t)4 * C * pad4(A::sdf(l).in) * 4));
        w.P[l] = reinterpret_cast<float*>(take((size_t)4 * C * pad4(A::sdf(l).out) * 4));
    }
    for (int l = 0; l < L::LC; ++l) {
        w.Xc[l] = reinterpret_cast<float*>(take((size_t)C * pad4(A::rgb(l).in) * 4));
        w.Pc[l] = reinterpret_cast<float*>(take((size_t)C * pad4(A::rgb(l).out) * 4));
    }
    w.bytes = (p - p0) + 256;
    return w;
}

// ---- the two passes over one chunk ---------------------------------------------------

// what one call of the layer-major path does: the backward from scratch (records and
// activations recomputed), the forward of a training step that keeps them in the
// workspace, or the backward from what that forward kept
enum class Pass { kBackward, kForwardKeep, kBackwardKept };

struct RenderOut {
    float* rgb;
    float* depth;
    float* wsum;
    float* normal;
    float* eik;
};

template <int ARCH>
int chunk_forward(cublasHandle_t h, const GemmWs<ARCH>& w, const NetParams& np, const SampleSource& src, int64_t c0,
                  int64_t n, cudaStream_t st) {
    using A = Arch<ARCH>;
    using L = GLayout<ARCH>;
    constexpr int E = A::kEnc;
    k_gsetup<<<grid_1d(n, kEw), kEw, 0, st>>>(np, src, c0, n, w.aux);
    k_genc<ARCH><<<grid_1d(n * pad4(E), kEw), kEw, 0, st>>>(w.aux, n, w.X[0]);
    int rc = cuda_check(cudaGetLastError(), "backward setup launch");
    if (rc) return rc;
    for (int l = 0; l < L::LS; ++l) {
        const Layer ly = A::sdf(l);
        const float* W = w.wp + L::sdf_off(l);
        rc = mm_fwd(h, 4 * n, pad4(ly.in), pad4(ly.out), w.X[l], pad4(ly.in), W, pad4(ly.in), w.P[l], pad4(ly.out));
        if (rc) return rc;
        const float* b = W + (int64_t)pad4(ly.out) * pad4(ly.in);
        if (l + 1 < L::LS) {
            const int ldn = pad4(A::sdf(l + 1).in);
            const bool skip = l + 1 == A::kSkip;
            k_gsp_fwd<<<grid_1d(n * ldn / 4, kEw), kEw, 0, st>>>(w.P[l], pad4(ly.out), b, ly.out, w.X[0], pad4(E), E, skip,
                                                             skip ? kSkipScale : 1.0f, np.beta, n, w.X[l + 1], ldn);
        } else {
            const int ldc = pad4(A::rgb(0).in);
            k_gsdf_out<ARCH><<<grid_1d(n * ldc, kEw), kEw, 0, st>>>(w.P[l], pad4(ly.out), b, w.aux, n, c0, np.scale,
                                                                     w.Xc[0], ldc, w.rec);
        }
        rc = cuda_check(cudaGetLastError(), "backward SDF activation launch");
        if (rc) return rc;
    }
    for (int l = 0; l < L::LC; ++l) {
        const Layer ly = A::rgb(l);
        const float* W = w.wp + L::rgb_off(l);
        rc = mm_fwd(h, n, pad4(ly.in), pad4(ly.out), w.Xc[l], pad4(ly.in), W, pad4(ly.in), w.Pc[l], pad4(ly.out));
        if (rc) return rc;
        const float* b = W + (int64_t)pad4(ly.out) * pad4(ly.in);
        if (l + 1 < L::LC) {
            const int ldn = pad4(A::rgb(l + 1).in);
            k_grelu_fwd<<<grid_1d(n * ldn / 4, kEw), kEw, 0, st>>>(w.Pc[l], pad4(ly.out), b, ly.out, n, w.Xc[l + 1], ldn);
        } else {
            k_grgb_out<<<grid_1d(n, kEw), kEw, 0, st>>>(w.Pc[l], pad4(ly.out), b, n, c0, w.rec);
        }
        rc = cuda_check(cudaGetLastError(), "backward colour activation launch");
        if (rc) return rc;
    }
    return TSDFS_OK;
}

template <int ARCH>
int chunk_backward(cublasHandle_t h, const GemmWs<ARCH>& w, const NetParams& np, int64_t c0, int64_t n, cudaStream_t st) {
    using A = Arch<ARCH>;
    using L = GLayout<ARCH>;
    // colour network, output layer first
    int rc;
    {
        const Layer ly = A::rgb(L::LC - 1);
        const float* b = w.wp + L::rgb_off(L::LC - 1) + (int64_t)pad4(ly.out) * pad4(ly.in);
        k_grgb_bwd<<<grid_1d(n, kEw), kEw, 0, st>>>(w.Pc[L::LC - 1], pad4(ly.out), b, w.adj, n, c0, w.G, pad4(ly.out));
        rc = cuda_check(cudaGetLastError(), "backward colour output launch");
        if (rc) return rc;
    }
    for (int l = L::LC - 1; l >= 0; --l) {
        const Layer ly = A::rgb(l);
        const int kp = pad4(ly.in), ldg = pad4(ly.out);
        const float* W = w.wp + L::rgb_off(l);
        float* dW = w.dwp + L::rgb_off(l);
        rc = mm_dw(h, n, ldg, kp, w.G, ldg, w.Xc[l], kp, dW, kp);
        if (!rc) rc = mv_db(h, n, ly.out, w.G, ldg, 1, w.ones, dW + (int64_t)ldg * kp);
        if (!rc) rc = mm_dx(h, n, ldg, kp, w.G, ldg, W, kp, w.D, kp);
        if (rc) return rc;
        if (l == 0) break;
        const Layer lp = A::rgb(l - 1);
        const float* bp = w.wp + L::rgb_off(l - 1) + (int64_t)pad4(lp.out) * pad4(lp.in);
        k_grelu_bwd<<<grid_1d(n * pad4(lp.out) / 4, kEw), kEw, 0, st>>>(w.D, kp, w.Pc[l - 1], pad4(lp.out), bp, lp.out, n,
                                                                   w.G, pad4(lp.out));
        rc = cuda_check(cudaGetLastError(), "backward ReLU launch");
        if (rc) return rc;
    }
    // w.D = adjoint of the colour input rows; the SDF output rows' adjoint
    {
        constexpr Layer lo = A::sdf(L::LS - 1);
        k_gsdf_out_bwd<ARCH><<<grid_1d(n * pad4(lo.out), kEw), kEw, 0, st>>>(w.D, pad4(A::rgb(0).in), w.adj, w.rec, n,
                                                                              c0, np.scale, w.G, pad4(lo.out));
        rc = cuda_check(cudaGetLastError(), "backward SDF output launch");
        if (rc) return rc;
    }
    for (int l = L::LS - 1; l >= 0; --l) {
        const Layer ly = A::sdf(l);
        const int kp = pad4(ly.in), ldg = pad4(ly.out);
        const float* W = w.wp + L::sdf_off(l);
        float* dW = w.dwp + L::sdf_off(l);
        rc = mm_dw(h, 4 * n, ldg, kp, w.G, ldg, w.X[l], kp, dW, kp);
        if (!rc) rc = mv_db(h, n, ly.out, w.G, ldg, 4, w.ones, dW + (int64_t)ldg * kp);
        if (rc) return rc;
        if (l == 0) break;
        rc = mm_dx(h, 4 * n, ldg, kp, w.G, ldg, W, kp, w.D, kp);
        if (rc) return rc;
        const Layer lp = A::sdf(l - 1);
        const float* bp = w.wp + L::sdf_off(l - 1) + (int64_t)pad4(lp.out) * pad4(lp.in);
        k_gsp_bwd<<<grid_1d(n * pad4(lp.out) / 4, kEw), kEw, 0, st>>>(w.D, kp, w.P[l - 1], pad4(lp.out), bp, lp.out,
                                                           l == A::kSkip ? kSkipScale : 1.0f, np.beta, n, w.G,
                                                           pad4(lp.out));
        rc = cuda_check(cudaGetLastError(), "backward softplus launch");
        if (rc) return rc;
    }
    return TSDFS_OK;
}

template <int ARCH>
int run(Pass pass, const tsdfs_mlp* mlp, const float* ray_o, const float* ray_d, const float* t_n, const float* t_f,
        const int32_t* offsets, const uint8_t* status, int64_t n_rays, int64_t max_samples, const float* d_rgb,
        const float* d_depth, const float* d_eik, float* d_sdf_w, float* d_rgb_w, const RenderOut& out, void* ws,
        size_t ws_bytes, cudaStream_t st) {
    using L = GLayout<ARCH>;
    GemmWs<ARCH> w = gemm_layout<ARCH>(ws, max_samples);
    if (!ws || ws_bytes < w.bytes) return fail(TSDFS_E_WORKSPACE, "layer-major workspace too small");
    const bool forward = pass == Pass::kForwardKeep;
    ProfScope ps(forward ? "train_forward" : "backward", st);
    // the sample total sizes the GEMMs
    int32_t total32 = 0;
    int rc = cuda_check(cudaMemcpyAsync(&total32, offsets + n_rays, sizeof(int32_t), cudaMemcpyDeviceToHost, st),
                        "layer-major total read");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "layer-major total sync");
    if (rc) return rc;
    const int64_t total = total32;
    const Opacity op{mlp->opacity, mlp->inv_s, mlp->alpha_eps};
    if (total > max_samples || total <= 0) {
        if (total > max_samples) {
            k_flag_overflow<<<1, 32, 0, st>>>(offsets + n_rays, max_samples, device_status_word());
            rc = cuda_check(cudaGetLastError(), "layer-major overflow flag");
            if (rc) return rc;
        }
        // no network work; the forward still writes its outputs (zero for an overflow, as render_rays)
        if (!forward) return TSDFS_OK;
        return launch_composite(w.rec, offsets, 0, status, n_rays, offsets + n_rays, max_samples, op, out.rgb,
                                out.depth, out.wsum, out.normal, out.eik, st);
    }
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

    std::lock_guard<std::mutex> lk(g_blas.mu);
    cublasHandle_t h = nullptr;
    rc = blas_handle(&h);
    if (rc) return rc;
    rc = blas_check(cublasSetStream(h, st), "set stream");
    if (!rc) rc = blas_check(cublasSetWorkspace(h, w.blas, kBlasWorkspace), "set workspace");
    if (rc) return rc;
    k_check_params<<<grid_1d(sdf_param_count<ARCH>() + rgb_param_count<ARCH>(), kEw), kEw, 0, st>>>(
        mlp->sdf_w, sdf_param_count<ARCH>(), mlp->rgb_w, rgb_param_count<ARCH>(), device_status_word());
    k_pad_weights<ARCH><<<grid_1d(L::total(), kEw), kEw, 0, st>>>(mlp->sdf_w, mlp->rgb_w, w.wp);
    rc = cuda_check(cudaGetLastError(), "layer-major weight copy launch");
    if (rc) return rc;
    const int64_t C = w.chunk;
    const int64_t last_c0 = (total - 1) / C * C;   // first sample of the last chunk
    // pass 1: the records of every sample, chunk by chunk; the last chunk's activations stay
    if (pass != Pass::kBackwardKept) {
        ProfScope pf(forward ? "train_forward_network" : "backward_forward", st);
        for (int64_t c0 = 0; c0 < total; c0 += C) {
            rc = chunk_forward<ARCH>(h, w, np, src, c0, total - c0 < C ? total - c0 : C, st);
            if (rc) return rc;
        }
    }
    if (forward) {
        ProfScope pc("train_forward_composite", st);
        return launch_composite(w.rec, offsets, 0, status, n_rays, offsets + n_rays, max_samples, op, out.rgb,
                                out.depth, out.wsum, out.normal, out.eik, st);
    }
    k_fill<<<grid_1d(w.chunk, kEw), kEw, 0, st>>>(w.ones, w.chunk, 1.0f);
    rc = cuda_check(cudaGetLastError(), "backward fill launch");
    if (!rc) rc = cuda_check(cudaMemsetAsync(w.dwp, 0, (size_t)L::total() * 4, st), "backward gradient clear");
    if (rc) return rc;
    {
        ProfScope pc("backward_composite", st);
        rc = launch_comp_bwd(w.rec, offsets, status, ray_d, n_rays, mlp, d_rgb, d_depth, d_eik, w.adj, st);
        if (rc) return rc;
    }
    {
        // the last chunk first, from the activations pass 1 left; the others recomputed
        ProfScope pn("backward_network", st);
        for (int64_t c0 = last_c0; c0 >= 0; c0 -= C) {
            const int64_t n = total - c0 < C ? total - c0 : C;
            if (c0 != last_c0) {
                rc = chunk_forward<ARCH>(h, w, np, src, c0, n, st);
                if (rc) return rc;
            }
            rc = chunk_backward<ARCH>(h, w, np, c0, n, st);
            if (rc) return rc;
        }
    }
    k_add_grads<ARCH><<<grid_1d(sdf_param_count<ARCH>() + rgb_param_count<ARCH>(), kEw), kEw, 0, st>>>(w.dwp, d_sdf_w,
                                                                                                       d_rgb_w);
    return cuda_check(cudaGetLastError(), "backward gradient add launch");
}

}  // namespace

size_t gemm_backward_workspace(const tsdfs_mlp* mlp, int64_t max_samples) {
    if (mlp->arch == TSDFS_ARCH_TINY) return gemm_layout<TSDFS_ARCH_TINY>(nullptr, max_samples).bytes + 256;
    return gemm_layout<TSDFS_ARCH_ROOM>(nullptr, max_samples).bytes + 256;
}

int64_t gemm_backward_chunk(const tsdfs_mlp* mlp, int64_t max_samples) {
    return mlp->arch == TSDFS_ARCH_TINY ? chunk_samples<TSDFS_ARCH_TINY>(max_samples)
                                        : chunk_samples<TSDFS_ARCH_ROOM>(max_samples);
}

int gemm_backward(const tsdfs_mlp* mlp, const float* ray_o, const float* ray_d, const float* t_n, const float* t_f,
                  const int32_t* offsets, const uint8_t* status, int64_t n_rays, int64_t max_samples,
                  const float* d_rgb, const float* d_depth, const float* d_eik, float* d_sdf_w, float* d_rgb_w,
                  void* ws, size_t ws_bytes, cudaStream_t st, bool kept) {
    const Pass pass = kept ? Pass::kBackwardKept : Pass::kBackward;
    const RenderOut none{};
    if (mlp->arch == TSDFS_ARCH_TINY)
        return run<TSDFS_ARCH_TINY>(pass, mlp, ray_o, ray_d, t_n, t_f, offsets, status, n_rays, max_samples, d_rgb,
                                    d_depth, d_eik, d_sdf_w, d_rgb_w, none, ws, ws_bytes, st);
    return run<TSDFS_ARCH_ROOM>(pass, mlp, ray_o, ray_d, t_n, t_f, offsets, status, n_rays, max_samples, d_rgb,
                                d_depth, d_eik, d_sdf_w, d_rgb_w, none, ws, ws_bytes, st);
}

int gemm_train_forward(const tsdfs_mlp* mlp, const float* ray_o, const float* ray_d, const float* t_n,
                       const float* t_f, const int32_t* offsets, const uint8_t* status, int64_t n_rays,
                       int64_t max_samples, float* rgb, float* depth, float* wsum, float* normal, float* eik, void* ws,
                       size_t ws_bytes, cudaStream_t st) {
    const RenderOut out{rgb, depth, wsum, normal, eik};
    if (mlp->arch == TSDFS_ARCH_TINY)
        return run<TSDFS_ARCH_TINY>(Pass::kForwardKeep, mlp, ray_o, ray_d, t_n, t_f, offsets, status, n_rays,
                                    max_samples, nullptr, nullptr, nullptr, nullptr, nullptr, out, ws, ws_bytes, st);
    return run<TSDFS_ARCH_ROOM>(Pass::kForwardKeep, mlp, ray_o, ray_d, t_n, t_f, offsets, status, n_rays, max_samples,
                                nullptr, nullptr, nullptr, nullptr, nullptr, out, ws, ws_bytes, st);
}

}  // namespace tsdfs
