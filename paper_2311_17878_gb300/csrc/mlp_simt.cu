// FP32 SIMT evaluation of the SDF and colour networks at ray samples.
//
// A CTA takes a tile of kTS samples.  The SDF gradient is carried in forward
// mode: each sample owns four rows [value; d/dx; d/dy; d/dz] that share every
// weight load; a hidden layer maps value rows through softplus_beta and
// tangent rows through its slope sigma(beta z) (1 on the linear branch).  The
// colour network then runs on one row per sample.  Activations live in shared
// memory (two ping-pong buffers); each layer's weights stream through a
// K-chunk tile in shared memory.  Results go to a per-sample record consumed
// by the compositing kernel.
#include "common.cuh"

namespace tsdfs {

namespace {

constexpr int kThreads = 256;
constexpr int kTS = 16;          // samples per tile (64 rows with tangents)
constexpr int kKC = 16;          // K chunk of a weight tile
constexpr int kLDA = 297;        // activation row stride (odd: no bank conflicts)
constexpr int kMaxNPad = 272;    // widest layer (257) padded to 16
constexpr int kLDW = kMaxNPad + 1;

struct Smem {
    float act[2][4 * kTS][kLDA];
    float wt[kKC][kLDW];
    float enc[4 * kTS][40];      // encoded input (and tangents), kept for the skip layer
    float xt[kTS][3];            // normalised position
    float dir[kTS][3];
    float tval[kTS], dval[kTS];
    int valid[kTS];
    long long ray[kTS];
};

__device__ __forceinline__ float softplus_b(float z, float beta) {
    const float bz = beta * z;
    return bz > 20.0f ? z : log1pf(expf(bz)) / beta;
}
__device__ __forceinline__ float softplus_slope(float z, float beta) {
    const float bz = beta * z;
    return bz > 20.0f ? 1.0f : 1.0f / (1.0f + expf(-bz));
}

// acc[r][j] = sum_k in[row(r)][k] * W[col(j)][k] for this thread's RPT rows and
// columns n = j*16 + cg (cg = thread % 16).  W is [N][K] row-major in global.
template <int K, int N, int RPT>
__device__ __forceinline__ void gemm(Smem& sm, const float (*in)[kLDA], int row0, const float* __restrict__ W,
                                     float (&acc)[RPT][(N + 15) / 16]) {
    constexpr int NJ = (N + 15) / 16;
    constexpr int NPAD = NJ * 16;
    const int cg = threadIdx.x & 15;
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
        for (int j = 0; j < NJ; ++j) acc[r][j] = 0.0f;
    for (int k0 = 0; k0 < K; k0 += kKC) {
        __syncthreads();
        for (int e = threadIdx.x; e < kKC * NPAD; e += kThreads) {
            const int kk = e % kKC, n = e / kKC;
            const int k = k0 + kk;
            sm.wt[kk][n] = (n < N && k < K) ? __ldg(W + (int64_t)n * K + k) : 0.0f;
        }
        __syncthreads();
        const int kmax = K - k0 < kKC ? K - k0 : kKC;
        for (int kk = 0; kk < kmax; ++kk) {
            float a[RPT];
#pragma unroll
            for (int r = 0; r < RPT; ++r) a[r] = in[row0 + r][k0 + kk];
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const float w = sm.wt[kk][j * 16 + cg];
#pragma unroll
                for (int r = 0; r < RPT; ++r) acc[r][j] = fmaf(a[r], w, acc[r][j]);
            }
        }
    }
}

// hidden SDF layer with forward-mode tangents: rows row0..row0+3 of one sample
template <int K, int N>
__device__ __forceinline__ void sdf_hidden(Smem& sm, int src, const float* __restrict__ W, const float* __restrict__ b,
                                           float beta, bool tangents) {
    constexpr int NJ = (N + 15) / 16;
    const int s = threadIdx.x >> 4, cg = threadIdx.x & 15;
    float acc[4][NJ];
    gemm<K, N, 4>(sm, sm.act[src], 4 * s, W, acc);
    float(*out)[kLDA] = sm.act[src ^ 1];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int n = j * 16 + cg;
        if (n < N) {
            const float z = acc[0][j] + __ldg(b + n);
            if (tangents) {
                out[4 * s][n] = softplus_b(z, beta);
                const float sl = softplus_slope(z, beta);
                out[4 * s + 1][n] = sl * acc[1][j];
                out[4 * s + 2][n] = sl * acc[2][j];
                out[4 * s + 3][n] = sl * acc[3][j];
            } else {
                // value-only tiles: the four rows are four samples
                out[4 * s][n] = softplus_b(z, beta);
                out[4 * s + 1][n] = softplus_b(acc[1][j] + __ldg(b + n), beta);
                out[4 * s + 2][n] = softplus_b(acc[2][j] + __ldg(b + n), beta);
                out[4 * s + 3][n] = softplus_b(acc[3][j] + __ldg(b + n), beta);
            }
        }
    }
}

template <int ARCH, bool TANGENTS>
__device__ void sdf_network(Smem& sm, const NetParams& np, int& cur) {
    using A = Arch<ARCH>;
    const float* w = np.sdf_w;
#define TSDFS_HID(L)                                                                                   \
    {                                                                                                  \
        constexpr Layer ly = A::sdf(L);                                                                \
        if (L == A::kSkip) {                                                                           \
            __syncthreads();                                                                           \
            for (int e = threadIdx.x; e < 4 * kTS * 256; e += kThreads) {                              \
                const int row = e >> 8, k = e & 255;                                                   \
                const int hw = 256 - A::kEnc;                                                          \
                float v = k < hw ? sm.act[cur][row][k] : sm.enc[row][k - hw];                          \
                sm.act[cur][row][k] = v * 0.70710678118654752f;                                        \
            }                                                                                          \
        }                                                                                              \
        const float* W = w + sdf_layer_offset<ARCH>(L);                                                \
        sdf_hidden<ly.in, ly.out>(sm, cur, W, W + (int64_t)ly.out * ly.in, np.beta, TANGENTS);        \
        cur ^= 1;                                                                                      \
    }
    TSDFS_HID(0)
    TSDFS_HID(1)
    TSDFS_HID(2)
    if constexpr (A::kSdfLayers == 8) {
        TSDFS_HID(3)
        TSDFS_HID(4)
        TSDFS_HID(5)
        TSDFS_HID(6)
    }
#undef TSDFS_HID
}

// Encode the tile's inputs: gamma(x~) (and its Jacobian rows) into act[0] and enc.
template <int ARCH, bool TANGENTS>
__device__ void encode_inputs(Smem& sm) {
    using A = Arch<ARCH>;
    constexpr int E = A::kEnc;
    const int rows_per = TANGENTS ? 4 : 1;
    const int nsamp = TANGENTS ? kTS : 4 * kTS;
    for (int e = threadIdx.x; e < nsamp * E; e += kThreads) {
        const int s = e / E, c = e % E;
        float xs[3];
        if (TANGENTS) {
            xs[0] = sm.xt[s][0]; xs[1] = sm.xt[s][1]; xs[2] = sm.xt[s][2];
        } else {
            // value-only tiles keep their positions in enc rows (filled by the caller)
            xs[0] = sm.enc[s][36]; xs[1] = sm.enc[s][37]; xs[2] = sm.enc[s][38];
        }
        float val, tan[3] = {0.0f, 0.0f, 0.0f};
        if (c < 3) {
            val = xs[c];
            tan[c] = 1.0f;
        } else {
            const int q = c - 3;
            const int oct = q / 6, part = (q % 6) / 3, a = q % 3;
            const float f = (float)(1 << oct);
            float sn, cs;
            sincosf(f * xs[a], &sn, &cs);
            val = part == 0 ? sn : cs;
            tan[a] = part == 0 ? f * cs : -f * sn;
        }
        if (TANGENTS) {
            sm.act[0][4 * s][c] = val;
            sm.act[0][4 * s + 1][c] = tan[0];
            sm.act[0][4 * s + 2][c] = tan[1];
            sm.act[0][4 * s + 3][c] = tan[2];
        } else {
            sm.act[0][s][c] = val;
        }
        (void)rows_per;
    }
    __syncthreads();
    if (A::kSkip >= 0) {
        const int rows = TANGENTS ? 4 * kTS : 4 * kTS;
        for (int e = threadIdx.x; e < rows * E; e += kThreads) {
            const int row = e / E, c = e % E;
            sm.enc[row][c] = sm.act[0][row][c];
        }
    }
    __syncthreads();
}

template <int K, int N, bool SIGMOID>
__device__ __forceinline__ void rgb_layer(Smem& sm, int src, const float* __restrict__ W, const float* __restrict__ b) {
    constexpr int NJ = (N + 15) / 16;
    const int s = threadIdx.x >> 4, cg = threadIdx.x & 15;
    float acc[1][NJ];
    gemm<K, N, 1>(sm, sm.act[src], s, W, acc);
    float(*out)[kLDA] = sm.act[src ^ 1];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int n = j * 16 + cg;
        if (n < N) {
            const float z = acc[0][j] + __ldg(b + n);
            out[s][n] = SIGMOID ? 1.0f / (1.0f + expf(-z)) : fmaxf(z, 0.0f);
        }
    }
}

template <int ARCH>
__device__ void rgb_network(Smem& sm, const NetParams& np, int& cur) {
    using A = Arch<ARCH>;
#define TSDFS_RGB(L, SIG)                                                            \
    {                                                                                \
        constexpr Layer ly = A::rgb(L);                                              \
        const float* W = np.rgb_w + rgb_layer_offset<ARCH>(L);                       \
        rgb_layer<ly.in, ly.out, SIG>(sm, cur, W, W + (int64_t)ly.out * ly.in);      \
        cur ^= 1;                                                                    \
    }
    TSDFS_RGB(0, false)
    TSDFS_RGB(1, false)
    if constexpr (A::kRgbLayers == 5) {
        TSDFS_RGB(2, false)
        TSDFS_RGB(3, false)
        TSDFS_RGB(4, true)
    } else {
        TSDFS_RGB(2, true)
    }
#undef TSDFS_RGB
}

// Full evaluation: f, grad f, colour for each sample -> records.
template <int ARCH>
__global__ void __launch_bounds__(kThreads, 1) k_mlp_full(NetParams np, SampleSource src, SampleRec* __restrict__ rec,
                                                          uint32_t* dev_status) {
    using A = Arch<ARCH>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    int64_t total = sample_total(src);
    if (total > src.capacity) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(dev_status, TSDFS_DEV_SAMPLES_OVERFLOW);
        return;
    }
    const int64_t n_tiles = (total + kTS - 1) / kTS;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        __syncthreads();
        if (threadIdx.x < kTS) {
            const int s = threadIdx.x;
            const int64_t g = tile * kTS + s;
            const bool ok = g < total;
            float t = 0.0f, dl = 0.0f;
            int64_t r = 0;
            if (ok) {
                if (src.mode == kUniform) {
                    r = find_ray(src.offsets, src.n_rays, g);
                    const int i = (int)(g - __ldg(src.offsets + r));
                    const int n = __ldg(src.offsets + r + 1) - __ldg(src.offsets + r);
                    const float tn = __ldg(src.t_n + r), tf = __ldg(src.t_f + r);
                    dl = (tf - tn) / (float)n;
                    t = tn + ((float)i + 0.5f) * dl;
                } else {
                    r = explicit_ray(src, g);
                    t = __ldg(src.t + g);
                    dl = __ldg(src.delta + g);
                }
            }
            float o[3], d[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                o[a] = ok ? __ldg(src.ray_o + 3 * r + a) : 0.0f;
                d[a] = ok ? __ldg(src.ray_d + 3 * r + a) : 0.0f;
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float x = o[a] + t * d[a];
                sm.xt[s][a] = (x - np.center[a]) * np.inv_scale;
                sm.dir[s][a] = d[a];
            }
            sm.tval[s] = t;
            sm.dval[s] = dl;
            sm.valid[s] = ok;
            sm.ray[s] = r;
        }
        __syncthreads();
        encode_inputs<ARCH, true>(sm);
        int cur = 0;
        sdf_network<ARCH, true>(sm, np, cur);
        // output layer: [net_0, feature] with tangents of net_0
        {
            constexpr Layer ly = A::sdf(A::kSdfLayers - 1);
            constexpr int NJ = (ly.out + 15) / 16;
            const float* W = np.sdf_w + sdf_layer_offset<ARCH>(A::kSdfLayers - 1);
            const float* b = W + (int64_t)ly.out * ly.in;
            const int s = threadIdx.x >> 4, cg = threadIdx.x & 15;
            float acc[4][NJ];
            gemm<ly.in, ly.out, 4>(sm, sm.act[cur], 4 * s, W, acc);
            __syncthreads();
            // colour input row s of the other buffer: [x~, dir enc, n^, feature]
            float(*out)[kLDA] = sm.act[cur ^ 1];
            constexpr int fo = 3 + A::kDirEnc + 3;
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const int n = j * 16 + cg;
                if (n >= 1 && n < ly.out) out[s][fo + n - 1] = acc[0][j] + __ldg(b + n);
            }
            if (cg == 0) {  // column 0 lives in j = 0 of thread cg = 0
                const float f = np.scale * (acc[0][0] + __ldg(b));
                const float gx = acc[1][0], gy = acc[2][0], gz = acc[3][0];
                const float gn = sqrtf(gx * gx + gy * gy + gz * gz);
                const float inv = gn > 0.0f ? 1.0f / gn : 0.0f;
                const float nx = gx * inv, ny = gy * inv, nz = gz * inv;
                out[s][3 + A::kDirEnc + 0] = nx;
                out[s][3 + A::kDirEnc + 1] = ny;
                out[s][3 + A::kDirEnc + 2] = nz;
                out[s][0] = sm.xt[s][0];
                out[s][1] = sm.xt[s][1];
                out[s][2] = sm.xt[s][2];
                const float dx = sm.dir[s][0], dy = sm.dir[s][1], dz = sm.dir[s][2];
                if (A::kPeDir == 0) {
                    out[s][3] = dx; out[s][4] = dy; out[s][5] = dz;
                } else {
                    const float dv[3] = {dx, dy, dz};
                    out[s][3] = dx; out[s][4] = dy; out[s][5] = dz;
                    for (int oct = 0; oct < A::kPeDir; ++oct) {
                        const float fr = (float)(1 << oct);
                        for (int a = 0; a < 3; ++a) {
                            float sn, cs;
                            sincosf(fr * dv[a], &sn, &cs);
                            out[s][3 + 3 + oct * 6 + a] = sn;
                            out[s][3 + 3 + oct * 6 + 3 + a] = cs;
                        }
                    }
                }
                // stash f and the gradient in the record fields now
                const int64_t g = tile * kTS + s;
                if (sm.valid[s]) {
                    SampleRec& R = rec[g];
                    R.f = f;
                    R.dd = gx * dx + gy * dy + gz * dz;
                    R.t = sm.tval[s];
                    R.delta = sm.dval[s];
                    R.gnorm = gn;
                    R.nx = nx; R.ny = ny; R.nz = nz; R.pad = 0.0f;
                }
            }
            cur ^= 1;
        }
        rgb_network<ARCH>(sm, np, cur);
        __syncthreads();
        if (threadIdx.x < kTS) {
            const int s = threadIdx.x;
            const int64_t g = tile * kTS + s;
            if (sm.valid[s]) {
                rec[g].r = sm.act[cur][s][0];
                rec[g].g = sm.act[cur][s][1];
                rec[g].b = sm.act[cur][s][2];
            }
        }
    }
}

// SDF values only (hierarchical coarse pass): 4*kTS samples per tile, one row each.
template <int ARCH>
__global__ void __launch_bounds__(kThreads, 1) k_mlp_value(NetParams np, SampleSource src, float* __restrict__ f_out,
                                                           uint32_t* dev_status) {
    using A = Arch<ARCH>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const int64_t total = sample_total(src);
    if (total > src.capacity) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(dev_status, TSDFS_DEV_SAMPLES_OVERFLOW);
        return;
    }
    constexpr int TS = 4 * kTS;
    const int64_t n_tiles = (total + TS - 1) / TS;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        __syncthreads();
        if (threadIdx.x < TS) {
            const int s = threadIdx.x;
            const int64_t g = tile * TS + s;
            const bool ok = g < total;
            int64_t r = 0;
            float t = 0.0f;
            if (ok) {
                if (src.mode == kUniform) {
                    r = src.sample_ray ? (int64_t)__ldg(src.sample_ray + g) : find_ray(src.offsets, src.n_rays, g);
                    const int i = (int)(g - __ldg(src.offsets + r));
                    const int n = __ldg(src.offsets + r + 1) - __ldg(src.offsets + r);
                    const float tn = __ldg(src.t_n + r), tf = __ldg(src.t_f + r);
                    const float dl = (tf - tn) / (float)n;
                    t = tn + ((float)i + 0.5f) * dl;
                } else {
                    r = explicit_ray(src, g);
                    t = __ldg(src.t + g);
                }
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float x = __ldg(src.ray_o + 3 * r + a) + t * __ldg(src.ray_d + 3 * r + a);
                sm.enc[s][36 + a] = (x - np.center[a]) * np.inv_scale;
            }
        }
        __syncthreads();
        encode_inputs<ARCH, false>(sm);
        int cur = 0;
        sdf_network<ARCH, false>(sm, np, cur);
        {
            constexpr Layer ly = A::sdf(A::kSdfLayers - 1);
            constexpr int NJ = (ly.out + 15) / 16;
            const float* W = np.sdf_w + sdf_layer_offset<ARCH>(A::kSdfLayers - 1);
            const float* b = W + (int64_t)ly.out * ly.in;
            const int s = threadIdx.x >> 4, cg = threadIdx.x & 15;
            float acc[4][NJ];
            gemm<ly.in, ly.out, 4>(sm, sm.act[cur], 4 * s, W, acc);
            if (cg == 0) {
                for (int r = 0; r < 4; ++r) {
                    const int64_t g = tile * TS + 4 * s + r;
                    if (g < total) f_out[g] = np.scale * (acc[r][0] + __ldg(b));
                }
            }
        }
    }
}

}  // namespace

size_t mlp_simt_smem() { return sizeof(Smem); }

template <int ARCH>
static int ensure_attrs() {
    static bool done[2] = {false, false};
    if (done[ARCH]) return TSDFS_OK;
    const int smem = (int)sizeof(Smem);
    int rc = cuda_check(cudaFuncSetAttribute(k_mlp_full<ARCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                        "mlp smem attribute");
    if (rc) return rc;
    rc = cuda_check(cudaFuncSetAttribute(k_mlp_value<ARCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                    "mlp smem attribute");
    if (rc) return rc;
    done[ARCH] = true;
    return TSDFS_OK;
}

static unsigned persistent_blocks(int64_t tiles) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (unsigned)(tiles < sms ? (tiles < 1 ? 1 : tiles) : sms);
}

// max_samples: host-side bound on the sample total (sizes the persistent grid)
template <int ARCH>
int launch_mlp_full_simt(const NetParams& np, const SampleSource& src, SampleRec* rec, int64_t max_samples,
                         cudaStream_t st) {
    int rc = ensure_attrs<ARCH>();
    if (rc) return rc;
    k_mlp_full<ARCH><<<persistent_blocks((max_samples + kTS - 1) / kTS), kThreads, sizeof(Smem), st>>>(
        np, src, rec, device_status_word());
    return cuda_check(cudaGetLastError(), "mlp launch");
}

template <int ARCH>
int launch_mlp_value_simt(const NetParams& np, const SampleSource& src, float* f_out, cudaStream_t st) {
    int rc = ensure_attrs<ARCH>();
    if (rc) return rc;
    k_mlp_value<ARCH><<<persistent_blocks((sample_bound(src) + 4 * kTS - 1) / (4 * kTS)), kThreads, sizeof(Smem), st>>>(
        np, src, f_out, device_status_word());
    return cuda_check(cudaGetLastError(), "mlp value launch");
}

template int launch_mlp_full_simt<TSDFS_ARCH_TINY>(const NetParams&, const SampleSource&, SampleRec*, int64_t, cudaStream_t);
template int launch_mlp_full_simt<TSDFS_ARCH_ROOM>(const NetParams&, const SampleSource&, SampleRec*, int64_t, cudaStream_t);
template int launch_mlp_value_simt<TSDFS_ARCH_TINY>(const NetParams&, const SampleSource&, float*, cudaStream_t);
template int launch_mlp_value_simt<TSDFS_ARCH_ROOM>(const NetParams&, const SampleSource&, float*, cudaStream_t);

}  // namespace tsdfs
