// Shared pieces of the tcgen05 network kernels: the layer tables of the packed
// 16-bit weights and the PTX helpers (mbarriers, 1-D bulk copies, tcgen05 MMA /
// TMEM loads, stmatrix, operand layout, activations).  Device code only.
#pragma once
#include <type_traits>

#include "common.cuh"

namespace tsdfs {
namespace {

constexpr int kKChunk = 64;                // K columns per weight chunk
constexpr uint32_t kMaxSpin = 1u << 26;    // bound of every mbarrier wait

struct TcLayer {
    int K, Kp, N, Np;
    bool sdf;
    int idx;          // index within its network
};

__host__ __device__ constexpr int pad16(int x) { return (x + 15) / 16 * 16; }
// column range [lo, hi) of a K-wide operand row written by column half hf:
// the split is rounded up to 16 so every 16-column block stays inside K
__host__ __device__ constexpr int half_lo(int K, int hf) { return hf ? pad16(K / 2) : 0; }
__host__ __device__ constexpr int half_hi(int K, int hf) { return hf ? K : pad16(K / 2); }
// the same for `parts` parts of whole 16-column blocks (K a multiple of 16)
__host__ __device__ constexpr int part_lo(int K, int pt, int parts) { return ((K / 16) * pt / parts) * 16; }
__host__ __device__ constexpr int part_hi(int K, int pt, int parts) { return pt + 1 == parts ? K : part_lo(K, pt + 1, parts); }
// the same in 8-column groups (K a multiple of 8): parts differ by at most one group, the
// last part (which also writes the skip input's encoding columns) being the smaller
__host__ __device__ constexpr int part8_lo(int K, int pt, int parts) { return ((K / 8) * pt + parts - 1) / parts * 8; }
__host__ __device__ constexpr int part8_hi(int K, int pt, int parts) { return pt + 1 == parts ? K : part8_lo(K, pt + 1, parts); }

// Layer tables of the packed 16-bit weights.  FOLD: the serial kernel's tables, in which
// the SDF output layer keeps only its value column net_0 and the colour network's first
// layer reads the last hidden SDF activation h directly: the feature columns
// feat = W_f h + b_f enter the colour network only through W_c,feat, so
// W_c,feat feat = (W_c,feat W_f) h + W_c,feat b_f, and the folded first colour layer has the
// inputs [h, x~, direction encoding, unit normal] with the weights
// [W_c,feat W_f | W_c,x | W_c,dir | W_c,n] and the bias b_c + W_c,feat b_f.  Its weights and
// the two folded layers' FP32 biases follow the unfolded layers in the packed buffer.
template <int ARCH, bool FOLD = false> struct TcArch {
    using A = Arch<ARCH>;
    using Plain = TcArch<ARCH, false>;
    static constexpr int kLayers = A::kSdfLayers + A::kRgbLayers;
    static constexpr int kLS = A::kSdfLayers;
    static constexpr int kH = A::sdf(A::kSdfLayers - 1).in;   // width of h, the last SDF layer's input
    static constexpr int kX = 3 + A::kDirEnc + 3;               // x~, direction encoding, unit normal
    static constexpr int kXp = pad16(kX);
    static_assert(kH % kKChunk == 0, "the folded colour input's h part fills whole weight chunks");
    __host__ __device__ static constexpr TcLayer layer(int L) {
        if (FOLD && L == kLS - 1) return TcLayer{kH, kH, 1, 16, true, L};
        if (FOLD && L == kLS) return TcLayer{kH + kX, kH + kXp, A::rgb(0).out, pad16(A::rgb(0).out), false, 0};
        if (L < A::kSdfLayers) {
            const Layer l = A::sdf(L);
            return TcLayer{l.in, pad16(l.in), l.out, pad16(l.out), true, L};
        }
        const Layer l = A::rgb(L - A::kSdfLayers);
        return TcLayer{l.in, pad16(l.in), l.out, pad16(l.out), false, L - A::kSdfLayers};
    }
    __host__ __device__ static constexpr bool folded(int L) { return FOLD && (L == kLS - 1 || L == kLS); }
    __host__ __device__ static constexpr int chunks(int L) { return (layer(L).Kp + kKChunk - 1) / kKChunk; }
    __host__ __device__ static constexpr int chunk_k(int L, int c) {
        return layer(L).Kp - c * kKChunk < kKChunk ? layer(L).Kp - c * kKChunk : kKChunk;
    }
    __host__ __device__ static constexpr int64_t chunk_bytes(int L, int c) { return (int64_t)layer(L).Np * chunk_k(L, c) * 2; }
    __host__ __device__ static constexpr int64_t layer_bytes(int L) {
        int64_t b = 0;
        for (int cc = 0; cc < chunks(L); ++cc) b += chunk_bytes(L, cc);
        return b;
    }
    // offset of chunk c of layer L in the packed buffer: the unfolded layers in order, then
    // (FOLD) the folded SDF output layer and the folded first colour layer
    __host__ __device__ static constexpr int64_t packed_offset(int L, int c) {
        int64_t off = 0;
        if (folded(L)) {
            off = Plain::packed_bytes();
            if (L == kLS) off += layer_bytes(kLS - 1);
        } else {
            for (int l = 0; l < L; ++l) off += Plain::layer_bytes(l);
        }
        for (int cc = 0; cc < c; ++cc) off += chunk_bytes(L, cc);
        return off;
    }
    // FP32 biases of the two folded layers (Np each), after their weights, 16-byte aligned
    __host__ __device__ static constexpr int64_t fold_bias_offset() {
        return (Plain::packed_bytes() + layer_bytes(kLS - 1) + layer_bytes(kLS) + 15) / 16 * 16;
    }
    __host__ __device__ static constexpr int fold_bias_count() { return layer(kLS - 1).Np + layer(kLS).Np; }
    __host__ __device__ static constexpr int64_t packed_bytes() {
        if constexpr (FOLD) return fold_bias_offset() + (int64_t)fold_bias_count() * 4;
        int64_t off = 0;
        for (int l = 0; l < kLayers; ++l) off += layer_bytes(l);
        return off;
    }
    __host__ __device__ static constexpr int64_t param_offset(int L) {
        return L < A::kSdfLayers ? sdf_layer_offset<ARCH>(L) : rgb_layer_offset<ARCH>(L - A::kSdfLayers);
    }
    // each layer's biases start on a 16-float boundary (zero padded to Np)
    __host__ __device__ static constexpr int bias_offset(int L) {
        int o = 0;
        for (int l = 0; l < L; ++l) o += layer(l).Np;
        return o;
    }
    __host__ __device__ static constexpr int bias_total() { return bias_offset(kLayers); }
    __host__ __device__ static constexpr uint32_t bias_bytes() { return (uint32_t)((bias_total() * 4 + 15) / 16 * 16); }
    __host__ __device__ static constexpr int total_chunks() { return chunk_index(kLayers, 0); }
    // per-tile weight-chunk schedule of the full kernel, built once per CTA: 12 bytes a chunk
    __host__ __device__ static constexpr uint32_t chunk_tab_bytes() { return (uint32_t)((total_chunks() * 12 + 15) / 16 * 16); }
    // index of chunk c of layer L within a tile's chunk sequence; chunks of the SDF layers
    __host__ __device__ static constexpr int chunk_index(int L, int c) {
        int j = 0;
        for (int l = 0; l < L; ++l) j += chunks(l);
        return j + c;
    }
    __host__ __device__ static constexpr int sdf_chunks() { return chunk_index(A::kSdfLayers, 0); }
    __host__ __device__ static constexpr int rgb_chunks() { return chunk_index(kLayers, 0) - sdf_chunks(); }
    __host__ __device__ static constexpr int64_t max_rgb_chunk_bytes() {
        int64_t m = 0;
        for (int l = A::kSdfLayers; l < kLayers; ++l)
            for (int c = 0; c < chunks(l); ++c) m = chunk_bytes(l, c) > m ? chunk_bytes(l, c) : m;
        return m;
    }
    __host__ __device__ static constexpr uint32_t stage_bytes() {
        int64_t m = 0;
        for (int l = 0; l < kLayers; ++l)
            for (int c = 0; c < chunks(l); ++c) m = chunk_bytes(l, c) > m ? chunk_bytes(l, c) : m;
        return (uint32_t)m;
    }
};

// --------------------------------------------------------------------------
// PTX helpers
// --------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; false on timeout or when another role aborted
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          uint32_t limit = kMaxSpin) {
    for (uint32_t it = 0;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255u) == 255u && *abort_flag) return false;
        if (it > limit) {
            *abort_flag = 1;
            return false;
        }
    }
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// shared -> global bulk copy (both addresses and the size 16-byte multiples), in this thread's
// bulk group; commit the group; wait until its sources have been read / until it completed
__device__ __forceinline__ void bulk_s2g(void* dst, uint32_t src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: no swizzle, K-major core matrices (8 rows x 16 B)
__device__ __forceinline__ uint64_t mdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;
}
// instruction descriptor: (BF16 | F16) x same -> FP32, both K-major
template <bool F16>
__host__ __device__ constexpr uint32_t idesc_mma(int M, int N) {
    return (1u << 4) | ((F16 ? 0u : 1u) << 7) | ((F16 ? 0u : 1u) << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// one lane of a converged warp (elect.sync); the MMA and commit forms below take it as a
// predicate, so the whole warp runs the issue loop and the descriptors stay warp-uniform
__device__ __forceinline__ uint32_t elect_one() {
    uint32_t e;
    asm volatile("{ .reg .pred q; elect.sync _|q, 0xffffffff; selp.u32 %0, 1, 0, q; }" : "=r"(e));
    return e;
}
__device__ __forceinline__ void mma_el(uint32_t el, uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{ .reg .pred p, q; setp.ne.b32 p, %4, 0; setp.ne.b32 q, %5, 0; @q tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc), "r"(el));
}
__device__ __forceinline__ void commit_el(uint32_t el, uint32_t bar) {
    asm volatile("{ .reg .pred q; setp.ne.b32 q, %1, 0; @q tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0]; }" ::"r"(bar), "r"(el) : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// 16 TMEM lanes x 16 columns (two 16x256b repetitions): thread t receives lane
// base + t/4 in registers 0, 1 (columns 2(t%4), 2(t%4)+1) and 4, 5 (the same
// columns + 8), and lane base + 8 + t/4 in registers 2, 3 and 6, 7
__device__ __forceinline__ void tmem_ld16x256_x2(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.16x256b.x2.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}
// one 16x256b repetition: 16 lanes x 8 columns, registers 0, 1 = lane base + t/4 and
// 2, 3 = lane base + 8 + t/4, at columns 2(t%4), 2(t%4)+1
__device__ __forceinline__ void tmem_ld16x256_x1(uint32_t taddr, float* v) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.16x256b.x1.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = __uint_as_float(r[j]);
}
// wait for this thread's TMEM loads; the registers they fill are operands, so no use of
// them can be scheduled before the wait
__device__ __forceinline__ void tmem_wait_ld16(float (&d)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3]), "+f"(d[4]), "+f"(d[5]), "+f"(d[6]), "+f"(d[7]),
                   "+f"(d[8]), "+f"(d[9]), "+f"(d[10]), "+f"(d[11]), "+f"(d[12]), "+f"(d[13]), "+f"(d[14]), "+f"(d[15])
                 :
                 : "memory");
}
// two 8x8 16-bit matrices: threads 0-15 give the row addresses (row i % 8 of matrix i / 8)
__device__ __forceinline__ void stmatrix2(uint32_t addr, uint32_t r0, uint32_t r1) {
    asm volatile("stmatrix.sync.aligned.m8n8.x2.shared.b16 [%0], {%1,%2};" ::"r"(addr), "r"(r0), "r"(r1) : "memory");
}
// four 8x8 16-bit matrices to shared memory: thread i supplies the address of row
// i % 8 of matrix i / 8; register j holds row t/4, columns 2(t%4), 2(t%4)+1 of matrix j
__device__ __forceinline__ void stmatrix4(uint32_t addr, uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3) {
    asm volatile("stmatrix.sync.aligned.m8n8.x4.shared.b16 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(r0), "r"(r1), "r"(r2),
                 "r"(r3)
                 : "memory");
}

// element (r, k) of a K-major no-swizzle operand with Kp columns -> byte offset
__device__ __forceinline__ uint32_t a_off(int r, int k, int Kp) {
    return (uint32_t)(((r >> 3) * (Kp >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}
template <bool F16>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    if constexpr (F16) {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
}
// max(x, 0) on both 16-bit halves of a packed pair; rounding is monotonic and keeps 0, so
// clamping after the rounding gives the value clamping before it would
template <bool F16>
__device__ __forceinline__ uint32_t relu2(uint32_t x) {
    if constexpr (F16) {
        __half2 h = __hmax2(*reinterpret_cast<__half2*>(&x), __float2half2_rn(0.0f));
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __nv_bfloat162 h = __hmax2(*reinterpret_cast<__nv_bfloat162*>(&x), __float2bfloat162_rn(0.0f));
        return *reinterpret_cast<uint32_t*>(&h);
    }
}
// store 8 consecutive columns (k0 multiple of 8) of row r
template <bool F16>
__device__ __forceinline__ void st_row8(uint8_t* base, int r, int k0, int Kp, const float* v) {
    uint4 q;
    q.x = pack2<F16>(v[0], v[1]);
    q.y = pack2<F16>(v[2], v[3]);
    q.z = pack2<F16>(v[4], v[5]);
    q.w = pack2<F16>(v[6], v[7]);
    *reinterpret_cast<uint4*>(base + a_off(r, k0, Kp)) = q;
}

// tanh on the special-function unit (max relative error about 2^-11)
__device__ __forceinline__ float tanh_fast(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// log(1 + u) on [0, 1]: degree-4 polynomial with p(0) = 0 and p(1) = ln 2 exactly,
// minimax-fitted (Lawson iteration) at Chebyshev nodes, |error| < 8e-5; divided by
// beta = 100 in the softplus this is below the FP16 rounding of the activations
// (fitted for this kernel; see the tests)
__device__ __forceinline__ float log1p_unit(float u) {
    float p = -0.05692862346768379f;
    p = fmaf(p, u, 0.22263112664222717f);
    p = fmaf(p, u, -0.4698040187358856f);
    p = fmaf(p, u, 0.9972487092018127f);
    return p * u;
}
// softplus_beta(z) and its slope sigma(beta z) from one tanh:
// t = tanh(beta z / 2); sigma(beta z) = (1 + t)/2; sigma(beta |z|) = (1 + |t|)/2 and
// softplus_beta(z) = max(z, 0) + log(1 + e^{-beta |z|})/beta = max(z, 0) + (ln 2 - log(1 + |t|))/beta
__device__ __forceinline__ void softplus_slope_tanh(float z, float half_beta, float inv_beta, float& h, float& sg) {
    const float t = tanh_fast(half_beta * z);
    sg = fmaf(0.5f, t, 0.5f);
    h = fmaxf(z, 0.0f) + (0.69314718055994531f - log1p_unit(fabsf(t))) * inv_beta;
}
// the same for two pre-activations at once in FP16 arithmetic, for the FP16-operand path
// (its activation and tangent rows are rounded to FP16 for the next layer anyway): one
// tanh.approx.f16x2 for both, the polynomial and the products in half2 (the correction
// term is below ln 2 / beta, so its FP16 rounding is below that of the activation)
__device__ __forceinline__ __half2 tanh_h2(__half2 x) {
    uint32_t xi = *reinterpret_cast<uint32_t*>(&x), yi;
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(yi) : "r"(xi));
    return *reinterpret_cast<__half2*>(&yi);
}
struct SoftplusH2 {
    __half2 half_beta, neg_inv_beta, ln2_inv_beta, c4, c3, c2, c1, half, zero;
};
__device__ __forceinline__ SoftplusH2 softplus_h2_consts(float half_beta, float inv_beta) {
    SoftplusH2 k;
    k.half_beta = __float2half2_rn(half_beta);
    k.neg_inv_beta = __float2half2_rn(-inv_beta);
    k.ln2_inv_beta = __float2half2_rn(0.69314718055994531f * inv_beta);
    k.c4 = __float2half2_rn(-0.05692862346768379f);
    k.c3 = __float2half2_rn(0.22263112664222717f);
    k.c2 = __float2half2_rn(-0.4698040187358856f);
    k.c1 = __float2half2_rn(0.9972487092018127f);
    k.half = __float2half2_rn(0.5f);
    k.zero = __float2half2_rn(0.0f);
    return k;
}
__device__ __forceinline__ void softplus_slope_h2(float z0, float z1, const SoftplusH2& k, __half2& h, __half2& sg) {
    const __half2 z = __floats2half2_rn(z0, z1);
    const __half2 t = tanh_h2(__hmul2(z, k.half_beta));
    sg = __hfma2(k.half, t, k.half);
    const __half2 u = __habs2(t);
    __half2 p = __hfma2(k.c4, u, k.c3);
    p = __hfma2(p, u, k.c2);
    p = __hfma2(p, u, k.c1);
    p = __hmul2(p, u);
    h = __hadd2(__hmax2(z, k.zero), __hfma2(p, k.neg_inv_beta, k.ln2_inv_beta));
}
__device__ __forceinline__ uint32_t h2u(__half2 v) { return *reinterpret_cast<uint32_t*>(&v); }

// f(std::integral_constant<int, I>{}) for I = B .. E - 1, expanded at compile time
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// positional encoding entry j of coordinate vector xt, and its derivative along axis a
__device__ __forceinline__ float enc_val(const float* xt, int j, int pe, int a, bool deriv) {
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

// the same entry from the per-tile tables: sx = the 3 coordinates, spe = sin / cos of
// 2^oct x_b at ((oct * 3 + b) * 2 + {0: sin, 1: cos}); comp 0 = value, comp a + 1 =
// derivative along axis a
__device__ __forceinline__ float enc_tab(const float* sx, const float* spe, int pe, int j, int comp) {
    if (j < 3) return comp == 0 ? sx[j] : (j == comp - 1 ? 1.0f : 0.0f);
    const int qq = j - 3;
    const int oct = qq / 6, part = (qq % 6) / 3, b = qq % 3;
    if (oct >= pe) return 0.0f;
    const float sn = spe[(oct * 3 + b) * 2], cs = spe[(oct * 3 + b) * 2 + 1];
    if (comp == 0) return part == 0 ? sn : cs;
    if (b != comp - 1) return 0.0f;
    const float f = (float)(1 << oct);
    return part == 0 ? f * cs : -f * sn;
}

}  // namespace
}  // namespace tsdfs
