// Shared device-side definitions of the CUDA path (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>
#include <mutex>

#include "tsdfs.h"

namespace tsdfs {

// ---------------------------------------------------------------------------
// host-side error reporting (abi.cu)
// ---------------------------------------------------------------------------
int fail(int code, const char* fmt, ...);
int cuda_check(cudaError_t e, const char* what);
// device status word of the current device (TSDFS_DEV_* bits), see abi.cu
uint32_t* device_status_word();
// cached device address of a __device__ variable in the current context: looked up
// again when the device's context has changed since the last lookup (after a
// cudaDeviceReset, for example)
struct SymbolCache {
    static constexpr int kDevices = 64;
    std::mutex mu;
    void* addr[kDevices] = {};
    unsigned long long ctx[kDevices] = {};
};
int symbol_address(SymbolCache& cache, const void* symbol, void** out, const char* what);
// test-only limits (tsdfs_set_test_limits): polls of a bounded mbarrier wait before it
// gives up (default kMaxSpin of the tensor-core kernels) and voxel steps of a ray walk
// (0: the grid's own bound nx + ny + nz + 8)
uint32_t test_spin_limit(uint32_t dflt);
int test_march_cap();
// test-only: the tensor-core kernels' producers stop before this weight chunk of each CTA's
// first tile (-1: never), so the MMA warp's wait for it runs out
int test_withhold_chunk();

// exclusive scan of n counts into offsets[0..n]; `sums` needs scan_chunks(n) + 1 ints (bounds.cu)
int64_t scan_chunks(int64_t n);
int exclusive_scan(const int32_t* cnt, int64_t n, int32_t* offsets, int32_t* sums, cudaStream_t st);

// kernel timing (tsdfs_profile): brackets the launches in its scope with events
void prof_begin(const char* name, cudaStream_t st, void** token);
void prof_end(void* token, cudaStream_t st);
struct ProfScope {
    void* token = nullptr;
    cudaStream_t st;
    ProfScope(const char* name, cudaStream_t s) : st(s) { prof_begin(name, s, &token); }
    ~ProfScope() { prof_end(token, st); }
};

// ---------------------------------------------------------------------------
// network architectures (the C ABI's TSDFS_ARCH_* tables)
// ---------------------------------------------------------------------------
struct Layer {
    int in, out;
};

template <int ARCH> struct Arch;

template <> struct Arch<TSDFS_ARCH_TINY> {
    static constexpr int kSdfLayers = 4;
    static constexpr int kRgbLayers = 3;
    static constexpr int kPeSdf = 0;
    static constexpr int kPeDir = 0;
    static constexpr int kSkip = -1;
    static constexpr int kFeat = 16;
    static constexpr int kEnc = 3;         // encoded SDF input width
    static constexpr int kDirEnc = 3;
    static constexpr int kWidth = 64;       // hidden width
    __host__ __device__ static constexpr Layer sdf(int l) {
        return l == 0 ? Layer{3, 64} : (l < 3 ? Layer{64, 64} : Layer{64, 17});
    }
    __host__ __device__ static constexpr Layer rgb(int l) {
        return l == 0 ? Layer{25, 64} : (l == 1 ? Layer{64, 64} : Layer{64, 3});
    }
};

template <> struct Arch<TSDFS_ARCH_ROOM> {
    static constexpr int kSdfLayers = 8;
    static constexpr int kRgbLayers = 5;
    static constexpr int kPeSdf = 6;
    static constexpr int kPeDir = 4;
    static constexpr int kSkip = 4;
    static constexpr int kFeat = 256;
    static constexpr int kEnc = 39;
    static constexpr int kDirEnc = 27;
    static constexpr int kWidth = 256;
    __host__ __device__ static constexpr Layer sdf(int l) {
        return l == 0 ? Layer{39, 256} : (l == 3 ? Layer{256, 217} : (l == 7 ? Layer{256, 257} : Layer{256, 256}));
    }
    __host__ __device__ static constexpr Layer rgb(int l) {
        return l == 0 ? Layer{289, 256} : (l == 4 ? Layer{256, 3} : Layer{256, 256});
    }
};

template <int ARCH> __host__ __device__ constexpr int64_t sdf_param_count() {
    int64_t n = 0;
    for (int l = 0; l < Arch<ARCH>::kSdfLayers; ++l) n += (int64_t)Arch<ARCH>::sdf(l).out * (Arch<ARCH>::sdf(l).in + 1);
    return n;
}
template <int ARCH> __host__ __device__ constexpr int64_t rgb_param_count() {
    int64_t n = 0;
    for (int l = 0; l < Arch<ARCH>::kRgbLayers; ++l) n += (int64_t)Arch<ARCH>::rgb(l).out * (Arch<ARCH>::rgb(l).in + 1);
    return n;
}
template <int ARCH> __host__ __device__ constexpr int64_t sdf_layer_offset(int l) {
    int64_t n = 0;
    for (int i = 0; i < l; ++i) n += (int64_t)Arch<ARCH>::sdf(i).out * (Arch<ARCH>::sdf(i).in + 1);
    return n;
}
template <int ARCH> __host__ __device__ constexpr int64_t rgb_layer_offset(int l) {
    int64_t n = 0;
    for (int i = 0; i < l; ++i) n += (int64_t)Arch<ARCH>::rgb(i).out * (Arch<ARCH>::rgb(i).in + 1);
    return n;
}

// ---------------------------------------------------------------------------
// per-sample record between the network kernels and compositing (workspace)
// ---------------------------------------------------------------------------
struct __align__(16) SampleRec {
    float f, dd, t, delta;      // SDF, v . grad f, sample position, section width
    float r, g, b, gnorm;       // colour, |grad f|
    float nx, ny, nz, pad;      // unit normal
};
static_assert(sizeof(SampleRec) == 48, "record layout");

// how the network kernel finds a sample's ray, t and delta
enum SampleMode : int {
    kUniform = 0,   // ragged offsets, midpoints of [t_n, t_f]
    kExplicit = 1,  // t[g], delta[g] given, ray = sample_ray[g] if given, else g / per_ray
};

struct NetParams {
    const float* sdf_w;
    const float* rgb_w;
    float center[3];
    float inv_scale, scale, beta;
};

struct SampleSource {
    int mode;
    const float* ray_o;
    const float* ray_d;
    // kUniform
    const int32_t* offsets;
    const float* t_n;
    const float* t_f;
    int64_t n_rays;
    const int32_t* sample_ray;  // optional: ray of every sample (else a binary search of offsets /
                                // g / per_ray)
    // kExplicit
    const float* t;
    const float* delta;
    int per_ray;
    // total sample count: *total_dev when given (uniform: = offsets[n_rays]), else total_host
    const int32_t* total_dev;
    int64_t total_host;
    int64_t capacity;  // records available in the workspace
};

// opacity of a sample's section (Eq. 1 with the backbone's SDF-to-density transform)
struct Opacity {
    int kind;     // TSDFS_OPACITY_NEUS / TSDFS_OPACITY_VOLSDF
    float inv_s;  // NeuS: s of Phi_s; VolSDF: a = 1 / beta (density scale and Laplace rate)
    float eps;    // NeuS ratio guard
};

__device__ __forceinline__ float sigmoid_acc(float x) { return 1.0f / (1.0f + expf(-x)); }

// VolSDF density sigma(f) = a Psi(-f), Psi the CDF of the zero-mean Laplace law of scale 1/a
__device__ __forceinline__ float laplace_density(float f, float a) {
    const float e = 0.5f * expf(-fabsf(f) * a);
    return a * (f >= 0.0f ? e : 1.0f - e);
}

// d sigma / d f = -a * (a / 2) exp(-a |f|)
__device__ __forceinline__ float laplace_density_slope(float f, float a) { return -0.5f * a * a * expf(-fabsf(f) * a); }

// opacity of the section of width dl around a sample of SDF f and slope dd = v . grad f
__device__ __forceinline__ float section_opacity(const Opacity& op, float f, float dd, float dl) {
    if (op.kind == TSDFS_OPACITY_VOLSDF) return -expm1f(-laplace_density(f, op.inv_s) * dl);
    const float c = fminf(dd, 0.0f);
    const float p_lo = sigmoid_acc(op.inv_s * (f - 0.5f * dl * c));
    const float p_hi = sigmoid_acc(op.inv_s * (f + 0.5f * dl * c));
    const float alpha = (p_lo - p_hi + op.eps) / (p_lo + op.eps);
    return fminf(fmaxf(alpha, 0.0f), 1.0f);
}

__device__ __forceinline__ int64_t sample_total(const SampleSource& s) {
    return s.total_dev ? (int64_t)__ldg(s.total_dev) : s.total_host;
}

// host-side upper bound on the sample total (sizes persistent grids)
inline int64_t sample_bound(const SampleSource& s) { return s.total_dev ? s.capacity : s.total_host; }

__device__ __forceinline__ int64_t explicit_ray(const SampleSource& s, int64_t g) {
    return s.sample_ray ? (int64_t)__ldg(s.sample_ray + g) : g / s.per_ray;
}

__device__ __forceinline__ int64_t find_ray(const int32_t* __restrict__ offsets, int64_t n_rays, int64_t g) {
    // largest r with offsets[r] <= g (offsets non-decreasing, offsets[0] = 0)
    int64_t lo = 0, hi = n_rays;  // invariant offsets[lo] <= g < offsets[hi]
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (__ldg(offsets + mid) <= g) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void set_status(uint32_t* status, uint32_t bits) {
    if (status) atomicOr(status, bits);
}

inline unsigned grid_1d(int64_t n, int block, int max_blocks = 152 * 32) {
    int64_t b = (n + block - 1) / block;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (unsigned)b;
}

}  // namespace tsdfs
