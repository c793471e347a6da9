// Pipelined tcgen05 evaluation of the SDF and colour networks.
//
// Tile: 32 samples = 128 operand rows.  TMEM lane quarter q holds samples
// 8q..8q+7 in four row groups of 8 lanes: the value rows (lanes 32q + 0..7),
// then the d/dx, d/dy and d/dz tangent rows of the same samples (forward-mode
// gradient, as in the 64-sample kernel of mlp_tc.cu).  One layer's accumulator
// is M = 128 x N <= 256 fp32, half of the 512 TMEM columns; consecutive layers
// alternate between the two halves.  That lets the next layer's MMAs run while
// the epilogue still works on this layer: the epilogue writes the next operand
// in 64-column blocks and signals each block on its own mbarrier, and the MMA
// warp starts a block's MMAs as soon as the block is written.  The weight chunks
// of a block stream through a ring of 1-D bulk copies, one producer warp per
// ring stage.
//
// Operand precisions (template MODE): FP16, BF16, or BF16 with every SDF layer's
// operand split into two BF16 parts, hi = bf16(x) and lo = bf16(x - hi), and
// two MMAs per K step into the same FP32 accumulator (the weights are BF16
// values, so hi * w + lo * w keeps about 16 significant bits of each activation);
// the colour layers use plain BF16 operands in that mode.
//
// The SDF output layer (1 + F outputs) runs as one MMA of N <= 256; a 257th
// output (the room network's last feature) is an FP32 dot product of the last
// hidden layer's activations with its weight row, accumulated by the epilogue
// that writes those activations.
//
// Warps 0-11 are the epilogue (warp w: TMEM lane quarter w % 4, column part
// w / 4; parts take the 8-column groups g with g % 3 == part, so every 64-column
// block fills at the same pace), warp 12 allocates TMEM and issues the MMAs
// (lane 0), warps 13.. stream weight chunks, one per ring stage.  Every wait is
// bounded; on timeout the kernel records TSDFS_DEV_TIMEOUT, drains its own
// copies and MMAs, frees TMEM and returns.
#include <type_traits>

#include "tc_common.cuh"

namespace tsdfs {

namespace {

constexpr int kPTile = 32;            // samples per tile
constexpr int kPEpiWarps = 12;        // 4 lane quarters x 3 column parts
constexpr int kPParts = 3;
constexpr int kPMmaWarp = 12;
constexpr int kPMaxBlocks = 5;        // 64-column operand blocks of the widest input (320 columns)
constexpr uint32_t kPABytes = 64 * 1024;        // 128 rows x 256 16-bit columns
constexpr uint32_t kPXMax = 128 * 64 * 2;       // the colour input beyond column 256 (<= 64 columns)
constexpr uint32_t kPBarBytes = 256;
constexpr int kPBatch = 4;            // 8-column groups an epilogue thread loads and computes together

template <int MODE> struct PipeMode {
    static constexpr bool kF16 = MODE == TSDFS_PREC_F16;
    static constexpr bool kSplit = MODE == TSDFS_PREC_BF16X2;
    // split operands take 128 KB of A; the plain modes have room for a third ring stage
    static constexpr int kStages = kSplit ? 2 : 3;
    static constexpr int kThreads = 32 * (kPMmaWarp + 1 + kStages);
};

template <int ARCH> struct PipeArch : TcArch<ARCH> {
    using TcArch<ARCH>::layer;
    using TcArch<ARCH>::kLayers;
    using TcArch<ARCH>::stage_bytes;
    using TcArch<ARCH>::bias_bytes;
    using TcArch<ARCH>::chunk_tab_bytes;
    using A = Arch<ARCH>;
    static constexpr int LS = A::kSdfLayers;
    // the SDF output layer's columns beyond 256 (at most one) come from the epilogue's dot product
    static constexpr bool kExtraCol = A::sdf(LS - 1).out > 256;
    static constexpr int kOutMma = A::sdf(LS - 1).out > 256 ? 256 : pad16(A::sdf(LS - 1).out);
    // colour input row: [x~ (3), direction encoding, unit normal (3), feature]; output column
    // oc of the SDF network (oc >= 1: feature oc - 1) sits at colour column oc + kD
    static constexpr int kD = 3 + A::kDirEnc + 3 - 1;
    static constexpr int kPitchX = layer(LS).Kp > 256 ? layer(LS).Kp - 256 : 0;
    __host__ __device__ static constexpr int pitch_main(int L) { return layer(L).Kp > 256 ? 256 : layer(L).Kp; }
    __host__ __device__ static constexpr int n_mma(int L) {
        return (L == LS - 1) ? kOutMma : (layer(L).Np > 256 ? 256 : layer(L).Np);
    }
    __host__ __device__ static constexpr uint32_t table_bytes() {
        return (uint32_t)(kPTile * (8 + 6 * (A::kPeSdf + A::kPeDir)) * 4);
    }
    // per-sample outputs kept for the record (8 floats), col 0 of the output rows (4 floats),
    // the partial dot products of the extra column (3 parts) and its weight row
    __host__ __device__ static constexpr uint32_t scratch_bytes() {
        return (uint32_t)((kPTile * 8 + 128 + kPParts * kPTile + (kExtraCol ? 256 : 0)) * 4);
    }
    template <int MODE> __host__ __device__ static constexpr size_t smem_bytes() {
        return kPABytes + (PipeMode<MODE>::kSplit ? kPABytes : kPXMax) + PipeMode<MODE>::kStages * (size_t)stage_bytes() +
               bias_bytes() + table_bytes() + scratch_bytes() + chunk_tab_bytes() + kPBarBytes;
    }
    template <int MODE> __host__ __device__ static constexpr bool valid() {
        bool ok = layer(LS).Kp <= 256 + 64 && kD % 8 == 0 && A::sdf(LS - 1).out <= 257;
        for (int l = 0; l < kLayers; ++l) {
            if (l != LS && layer(l).Kp > 256) ok = false;
            if (l != LS - 1 && layer(l).Np > 256) ok = false;
        }
        return ok;
    }
};

struct PChunk {
    uint32_t off, bytes;
    uint16_t slot, kc;
};
static_assert(sizeof(PChunk) == 12, "chunk table entry");

struct PipeParams {
    const uint8_t* packed;
    const float* sdf_w;
    const float* rgb_w;
    float center[3];
    float inv_scale, scale, beta;
    SampleSource src;
    SampleRec* rec;
    uint32_t* status;
    uint32_t spin;   // polls of a bounded wait before it gives up
    int withhold;    // test-only: weight chunk of the first tile whose copy is never issued (-1: none)
};

// one TMEM lane per thread, 1 or 4 consecutive columns
__device__ __forceinline__ void tmem_ld32x1(uint32_t taddr, float& v) {
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
    v = __uint_as_float(r);
}
__device__ __forceinline__ void tmem_ld32x4(uint32_t taddr, float (&v)[4]) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = __uint_as_float(r[j]);
}
// one 8x8 16-bit matrix: threads 0-7 give the row addresses; thread t's register holds
// row t / 4, columns 2 (t % 4) and 2 (t % 4) + 1
__device__ __forceinline__ void stmatrix1(uint32_t addr, uint32_t r0) {
    asm volatile("stmatrix.sync.aligned.m8n8.x1.shared.b16 [%0], {%1};" ::"r"(addr), "r"(r0) : "memory");
}
// wait for this thread's TMEM loads; the registers are operands so no use moves above it
__device__ __forceinline__ void tmem_wait_ld8(float (&d)[8]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3]), "+f"(d[4]), "+f"(d[5]), "+f"(d[6]), "+f"(d[7])
                 :
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_ld4(float (&d)[4]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3]) : : "memory");
}
// a split pair: hi = bf16(x), lo = bf16(x - hi), packed two columns at a time
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

template <int ARCH, int MODE>
__global__ void __launch_bounds__(PipeMode<MODE>::kThreads, 1) k_mlp_pipe(PipeParams p) {
    using TA = PipeArch<ARCH>;
    using A = Arch<ARCH>;
    using PM = PipeMode<MODE>;
    constexpr bool F16 = PM::kF16;
    constexpr bool kSplit = PM::kSplit;
    constexpr int kStages = PM::kStages;
    constexpr int NL = TA::kLayers;
    constexpr int LS = A::kSdfLayers;
    constexpr uint32_t kStage = TA::stage_bytes();
    constexpr int kNT = TA::total_chunks();
    static_assert(TA::template valid<MODE>(), "network shape outside the pipelined kernel's layout");
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* A_hi = smem;
    uint8_t* A_lo = smem + kPABytes;                       // split mode: the low parts
    uint8_t* X = smem + kPABytes;                          // colour input beyond column 256
    uint8_t* stage_base = smem + kPABytes + (kSplit ? kPABytes : kPXMax);
    float* sbias = reinterpret_cast<float*>(stage_base + kStages * kStage);
    float* s_x = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(sbias) + TA::bias_bytes());
    float* s_pe = s_x + kPTile * 8;
    float* s_pd = s_pe + kPTile * A::kPeSdf * 6;
    float* s_out = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(s_x) + TA::table_bytes());
    float* s_g = s_out + kPTile * 8;
    float* s_f255 = s_g + 128;
    float* s_w255 = s_f255 + kPParts * kPTile;
    PChunk* s_chunks = reinterpret_cast<PChunk*>(reinterpret_cast<uint8_t*>(s_out) + TA::scratch_bytes());
    uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(s_chunks) + TA::chunk_tab_bytes());
    // bars: full[kStages], empty[kStages], accf[2], ablk[kPMaxBlocks], epi, drain
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 2 + kPMaxBlocks + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const uint32_t bar_full0 = smem_u32(bars), bar_empty0 = smem_u32(bars + kStages);
    const uint32_t bar_accf0 = smem_u32(bars + 2 * kStages);
    const uint32_t bar_blk0 = smem_u32(bars + 2 * kStages + 2);
    const uint32_t bar_epi = smem_u32(bars + 2 * kStages + 2 + kPMaxBlocks);
    const uint32_t bar_drain = bar_epi + 8;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const int64_t total = sample_total(p.src);
    if (total > p.src.capacity) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(p.status, TSDFS_DEV_SAMPLES_OVERFLOW);
        return;
    }
    const int64_t n_tiles = (total + kPTile - 1) / kPTile;
    if ((int64_t)blockIdx.x >= n_tiles) return;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(bar_full0 + 8 * i, 1);
            mbar_init(bar_empty0 + 8 * i, 1);
        }
        mbar_init(bar_accf0, 1);
        mbar_init(bar_accf0 + 8, 1);
        for (int b = 0; b < kPMaxBlocks; ++b) mbar_init(bar_blk0 + 8 * b, kPEpiWarps);
        mbar_init(bar_epi, kPEpiWarps);
        mbar_init(bar_drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        uint32_t off = 0;
        for (int L = 0, j = 0; L < NL; ++L)
            for (int c = 0; c < TA::chunks(L); ++c, ++j) {
                s_chunks[j] = PChunk{off, (uint32_t)TA::chunk_bytes(L, c), (uint16_t)(j % kStages),
                                     (uint16_t)TA::chunk_k(L, c)};
                off += (uint32_t)TA::chunk_bytes(L, c);
            }
    }
    for (int i = threadIdx.x; i < TA::bias_total(); i += PM::kThreads) {
        int L = 0;
        while (L + 1 < NL && TA::bias_offset(L + 1) <= i) ++L;
        const TcLayer ly = TA::layer(L);
        const float* W = (ly.sdf ? p.sdf_w : p.rgb_w) + TA::param_offset(L);
        const int j = i - TA::bias_offset(L);
        sbias[i] = j < ly.N ? __ldg(W + (int64_t)ly.N * ly.K + j) : 0.0f;
    }
    if constexpr (TA::kExtraCol) {
        const TcLayer lo = TA::layer(LS - 1);
        for (int i = threadIdx.x; i < 256; i += PM::kThreads)
            s_w255[i] = i < lo.K ? __ldg(p.sdf_w + TA::param_offset(LS - 1) + (int64_t)256 * lo.K + i) : 0.0f;
    }
    if constexpr (!kSplit) {
        // the tangent rows of the colour input beyond column 256 are never written: clear them
        // once so that the rows the colour MMAs compute and the epilogue ignores stay finite
        for (int i = threadIdx.x; i < (int)(kPXMax / 16); i += PM::kThreads)
            reinterpret_cast<uint4*>(X)[i] = make_uint4(0, 0, 0, 0);
    } else {
        for (int i = threadIdx.x; i < (int)(kPABytes / 16); i += PM::kThreads)
            reinterpret_cast<uint4*>(A_lo)[i] = make_uint4(0, 0, 0, 0);
    }
    if (warp == kPMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp > kPMmaWarp) {
        // ------------------------------------------------ producers, one per ring stage
        if (lane == 0 && warp - kPMmaWarp - 1 < kStages) {
            const uint32_t own = (uint32_t)(warp - kPMmaWarp - 1);
            const uint32_t dst = smem_u32(stage_base + own * kStage);
            uint32_t issued = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
                for (int j = (int)own; j < kNT; j += kStages) {
                    // test-only: stop before the withheld chunk of the first tile
                    if (tile == blockIdx.x && j == p.withhold) { ok = false; break; }
                    const PChunk ci = s_chunks[j];
                    if (!mbar_wait(bar_empty0 + 8 * own, (issued & 1u) ^ 1u, abort_flag, p.spin)) { ok = false; break; }
                    mbar_expect_tx(bar_full0 + 8 * own, ci.bytes);
                    bulk_g2s(dst, p.packed + ci.off, ci.bytes, bar_full0 + 8 * own);
                    ++issued;
                }
            }
            if (!ok && issued > 0) {
                for (uint32_t it = 0; it < kMaxSpin && !mbar_try(bar_full0 + 8 * own, (issued - 1) & 1u); ++it) {
                }
            }
        }
    } else if (warp == kPMmaWarp) {
        // ---------------------------------------------------------------- MMA issuer: the
        // whole warp runs the loop (converged: the descriptors stay warp-uniform), one elected
        // lane issues the MMAs and commits
        {
            const uint32_t el = elect_one();
            uint32_t full_uses[kStages], blk_uses[kPMaxBlocks];
#pragma unroll
            for (int i = 0; i < kStages; ++i) full_uses[i] = 0;
#pragma unroll
            for (int i = 0; i < kPMaxBlocks; ++i) blk_uses[i] = 0;
            uint32_t lc = 0;
            bool ok = true;
            const uint32_t a_hi = smem_u32(A_hi), a_lo = smem_u32(A_lo), a_x = smem_u32(X);
            for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
                int j = 0;
                for (int L = 0; L < NL && ok; ++L, ++lc) {
                    const TcLayer ly = TA::layer(L);
                    const uint32_t d_tmem = tmem + (lc & 1u) * 256u;
                    const uint32_t idesc = idesc_mma<F16>(128, TA::n_mma(L));
                    const uint32_t a_sbo = (uint32_t)(TA::pitch_main(L) / 8) * 128u;
                    const bool two = kSplit && ly.sdf;
                    for (int c = 0; c < TA::chunks(L); ++c, ++j) {
                        uint32_t bph = 0;
#pragma unroll
                        for (int i = 0; i < kPMaxBlocks; ++i)
                            if (i == c) bph = blk_uses[i]++ & 1u;
                        if (!__all_sync(0xffffffffu, mbar_wait(bar_blk0 + 8 * c, bph, abort_flag, p.spin))) { ok = false; break; }
                        const PChunk ci = s_chunks[j];
                        uint32_t fph = 0;
#pragma unroll
                        for (int i = 0; i < kStages; ++i)
                            if ((uint32_t)i == ci.slot) fph = full_uses[i]++ & 1u;
                        if (!__all_sync(0xffffffffu, mbar_wait(bar_full0 + 8 * ci.slot, fph, abort_flag, p.spin))) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t b0 = smem_u32(stage_base + ci.slot * kStage);
                        const uint32_t b_sbo = (uint32_t)(ci.kc / 8) * 128u;
                        // descriptors built once per chunk (a chunk lies wholly below or above
                        // column 256) and advanced by 16 (256 bytes) per K step
                        const int k0 = c * kKChunk;
                        uint64_t bd = mdesc(b0, 128, b_sbo);
                        if (k0 < 256) {
                            const uint32_t ko = (uint32_t)(k0 / 8) * 128u;
                            uint64_t ah = mdesc(a_hi + ko, 128, a_sbo), al = mdesc(a_lo + ko, 128, a_sbo);
                            for (int kk = 0; kk < ci.kc / 16; ++kk) {
                                mma_el(el, d_tmem, ah, bd, idesc, (k0 | kk) != 0 ? 1u : 0u);
                                if (two) mma_el(el, d_tmem, al, bd, idesc, 1u);
                                ah += 16;
                                al += 16;
                                bd += 16;
                            }
                        } else {
                            uint64_t ax = mdesc(a_x + (uint32_t)((k0 - 256) / 8) * 128u, 128, (uint32_t)(TA::kPitchX / 8) * 128u);
                            for (int kk = 0; kk < ci.kc / 16; ++kk) {
                                mma_el(el, d_tmem, ax, bd, idesc, 1u);
                                ax += 16;
                                bd += 16;
                            }
                        }
                        commit_el(el, bar_empty0 + 8 * ci.slot);
                    }
                    if (!ok) break;
                    commit_el(el, bar_accf0 + 8 * (lc & 1u));
                }
            }
            if (!ok && el) {
                mma_commit(bar_drain);
                for (uint32_t it = 0; it < kMaxSpin && !mbar_try(bar_drain, 0); ++it) {
                }
            }
        }
    } else {
        // ------------------------------------------------------------------ epilogue
        const int q = warp & 3, pt = warp >> 2;
        const int sq = lane >> 2, fc = 2 * (lane & 3);   // sample within the quarter, column pair
        const int s = 8 * q + sq;                          // sample within the tile
        const uint32_t lq = (uint32_t)(32 * q) << 16, lq16 = (uint32_t)(32 * q + 16) << 16;
        const float half_beta = 0.5f * p.beta, inv_beta = 1.0f / p.beta;
        constexpr float kInvSqrt2 = 0.70710678118654752f;
        const SoftplusH2 spk = softplus_h2_consts(half_beta, inv_beta);
        const __half2 inv_sqrt2_h2 = __float2half2_rn(kInvSqrt2);
        const int et = threadIdx.x;
        uint32_t acc_uses[2] = {0, 0}, epi_ph = 0, lc = 0;
        bool ok = true;
        auto epi_sync = [&]() -> bool {
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_epi);
            const bool w = mbar_wait(bar_epi, epi_ph & 1u, abort_flag, p.spin);
            ++epi_ph;
            return __all_sync(0xffffffffu, w);
        };
        // operand writes of this warp for block b are done: make them visible to the MMAs
        auto block_done = [&](int b) {
            fence_proxy_async();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_blk0 + 8 * b);
        };
        // row address of A row 32q + lane (stmatrix: lane i gives row i of the four 8x8 matrices)
        auto row_addr = [&](uint8_t* base, int pitch) -> uint32_t { return smem_u32(base) + a_off(32 * q + lane, 0, pitch); };
        // a value / d-dx / d-dy / d-dz quadruple of 8-column groups: hi (and lo) operand parts
        auto store4 = [&](uint32_t ra_hi, uint32_t ra_lo, int c, const float (&v)[8], bool split) {
            const uint32_t co = (uint32_t)(c >> 3) * 128u;
            if (split) {
                uint32_t hi[4], lo[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) split2(v[2 * j], v[2 * j + 1], hi[j], lo[j]);
                stmatrix4(ra_hi + co, hi[0], hi[1], hi[2], hi[3]);
                stmatrix4(ra_lo + co, lo[0], lo[1], lo[2], lo[3]);
            } else {
                stmatrix4(ra_hi + co, pack2<F16>(v[0], v[1]), pack2<F16>(v[2], v[3]), pack2<F16>(v[4], v[5]),
                          pack2<F16>(v[6], v[7]));
            }
        };
        // the tile's sample table: x~, direction, t, delta, then sin / cos of the encodings
        auto build_table = [&](int64_t tile) -> bool {
            if (et < kPTile) {
                const int64_t g = tile * kPTile + et;
                float t = 0.0f, dl = 0.0f, xs[3] = {0.0f, 0.0f, 0.0f}, ds[3] = {0.0f, 0.0f, 0.0f};
                if (g < total) {
                    int64_t ray;
                    if (p.src.mode == kUniform) {
                        ray = p.src.sample_ray ? (int64_t)__ldg(p.src.sample_ray + g) : find_ray(p.src.offsets, p.src.n_rays, g);
                        const int32_t o0 = __ldg(p.src.offsets + ray), o1 = __ldg(p.src.offsets + ray + 1);
                        const float tn = __ldg(p.src.t_n + ray), tf = __ldg(p.src.t_f + ray);
                        dl = (tf - tn) / (float)(o1 - o0);
                        t = tn + ((float)(g - o0) + 0.5f) * dl;
                    } else {
                        ray = explicit_ray(p.src, g);
                        t = __ldg(p.src.t + g);
                        dl = __ldg(p.src.delta + g);
                    }
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        ds[a] = __ldg(p.src.ray_d + 3 * ray + a);
                        xs[a] = (__ldg(p.src.ray_o + 3 * ray + a) + t * ds[a] - p.center[a]) * p.inv_scale;
                    }
                }
                float* sx = s_x + et * 8;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    sx[a] = xs[a];
                    sx[3 + a] = ds[a];
                }
                sx[6] = t;
                sx[7] = dl;
            }
            if (!epi_sync()) return false;
            // sin / cos per (sample, axis, encoding): one sincos at octave 0, then the angle
            // doubled per octave (sin 2x = 2 sin x cos x, cos 2x = (cos x - sin x)(cos x + sin x))
            if (et < 6 * kPTile) {
                const int sm = et / 6, a = (et >> 1) % 3, which = et & 1;
                const int n_oct = which ? A::kPeDir : A::kPeSdf;
                float* dst = which ? s_pd + (sm * A::kPeDir * 3 + a) * 2 : s_pe + (sm * A::kPeSdf * 3 + a) * 2;
                if (n_oct > 0) {
                    float sn, cs;
                    sincosf(s_x[sm * 8 + 3 * which + a], &sn, &cs);
                    for (int oct = 0; oct < n_oct; ++oct) {
                        dst[oct * 6] = sn;
                        dst[oct * 6 + 1] = cs;
                        const float s2 = 2.0f * sn * cs, c2 = (cs - sn) * (cs + sn);
                        sn = s2;
                        cs = c2;
                    }
                }
            }
            return epi_sync();
        };
        // layer 0's input from the table: the encoding and its Jacobian rows
        auto write_input0 = [&]() {
            constexpr int Kp0 = TA::layer(0).Kp;
            const uint32_t ra_hi = row_addr(A_hi, Kp0), ra_lo = row_addr(A_lo, Kp0);
            const float* sx = s_x + s * 8;
            const float* sp = s_pe + s * A::kPeSdf * 6;
            for (int g = pt; g < Kp0 / 8; g += kPParts) {
                float v[8];
#pragma unroll
                for (int cp = 0; cp < 4; ++cp)
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int jj = 8 * g + fc + e;
                        v[2 * cp + e] = jj < A::kEnc ? enc_tab(sx, sp, A::kPeSdf, jj, cp) : 0.0f;
                    }
                store4(ra_hi, ra_lo, 8 * g, v, kSplit);
            }
            block_done(0);
        };

        ok = build_table(blockIdx.x);
        if (ok) write_input0();
        for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
            int boff = 0;
            for (int L = 0; L < NL; ++L, ++lc) {
                const TcLayer ly = TA::layer(L);
                const uint32_t hsel = lc & 1u;
                const bool w_ok = mbar_wait(bar_accf0 + 8 * hsel, acc_uses[hsel] & 1u, abort_flag, p.spin);
                ++acc_uses[hsel];
                if (!__all_sync(0xffffffffu, w_ok)) { ok = false; break; }
                tc_fence_after();
                const uint32_t th = tmem + hsel * 256u;
                const float* bias = sbias + boff;
                boff += ly.Np;
                if (ly.sdf && ly.idx < LS - 1) {
                    // ---- hidden SDF layer: softplus and its slope times the tangents ----
                    const int Kn = TA::layer(L + 1).Kp;
                    const bool skip_next = ly.idx + 1 == A::kSkip;
                    const float sc = skip_next ? kInvSqrt2 : 1.0f;
                    const bool dot = TA::kExtraCol && ly.idx == LS - 2;
                    const uint32_t ra_hi = row_addr(A_hi, Kn), ra_lo = row_addr(A_lo, Kn);
                    const float* sx = s_x + s * 8;
                    const float* sp = s_pe + s * A::kPeSdf * 6;
                    float part = 0.0f;   // dot product of the value row with the extra column's weights
                    const int ng = Kn / 8, nblk = (ng + 7) / 8;
                    const int n_full = ly.N / 8;   // groups wholly inside the layer's outputs
                    // one group: value, d/dx, d/dy, d/dz of sample s at columns c + fc, c + fc + 1
                    auto group = [&](int c, const float (&d)[8]) {
                        float v[8];
                        if (c + 8 <= ly.N) {
                            const float2 bb = *reinterpret_cast<const float2*>(bias + c + fc);
                            if constexpr (F16) {
                                // FP16 operands: softplus, slope and tangent products in half2 (the
                                // results are FP16 operands of the next layer either way)
                                __half2 h, sg;
                                softplus_slope_h2(d[0] + bb.x, d[1] + bb.y, spk, h, sg);
                                if (dot) {
                                    const float2 hf = __half22float2(h);
                                    part = fmaf(hf.x, s_w255[c + fc], fmaf(hf.y, s_w255[c + fc + 1], part));
                                }
                                if (skip_next) {
                                    sg = __hmul2(sg, inv_sqrt2_h2);
                                    h = __hmul2(h, inv_sqrt2_h2);
                                }
                                const uint32_t co = (uint32_t)(c >> 3) * 128u;
                                stmatrix4(ra_hi + co, h2u(h), h2u(__hmul2(sg, __floats2half2_rn(d[2], d[3]))),
                                          h2u(__hmul2(sg, __floats2half2_rn(d[4], d[5]))),
                                          h2u(__hmul2(sg, __floats2half2_rn(d[6], d[7]))));
                                return;
                            } else {
#pragma unroll
                                for (int e = 0; e < 2; ++e) {
                                    float h, sg;
                                    softplus_slope_tanh(d[e] + (e ? bb.y : bb.x), half_beta, inv_beta, h, sg);
                                    if (dot) part = fmaf(h, s_w255[c + fc + e], part);
                                    sg *= sc;
                                    v[e] = h * sc;
                                    v[2 + e] = sg * d[2 + e];
                                    v[4 + e] = sg * d[4 + e];
                                    v[6 + e] = sg * d[6 + e];
                                }
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                const int col = c + fc + e;
                                if (col < ly.N) {
                                    float h, sg;
                                    softplus_slope_tanh(d[e] + bias[col], half_beta, inv_beta, h, sg);
                                    if (dot) part = fmaf(h, s_w255[col], part);
                                    sg *= sc;
                                    v[e] = h * sc;
                                    v[2 + e] = sg * d[2 + e];
                                    v[4 + e] = sg * d[4 + e];
                                    v[6 + e] = sg * d[6 + e];
                                } else {
                                    // beyond the layer's outputs: the skip input gamma(x~) / sqrt(2), or zeros
                                    const int en = col - ly.N;
                                    float val = 0.0f, der = 0.0f;
                                    int ax = -1;
                                    if (skip_next && en < A::kEnc) {
                                        if (en < 3) {
                                            ax = en;
                                            val = sx[en];
                                            der = 1.0f;
                                        } else {
                                            const int qq = en - 3, oct = qq / 6, prt = (qq % 6) / 3;
                                            ax = qq % 3;
                                            const float sn = sp[(oct * 3 + ax) * 2], cs = sp[(oct * 3 + ax) * 2 + 1];
                                            const float f = (float)(1 << oct);
                                            val = prt == 0 ? sn : cs;
                                            der = prt == 0 ? f * cs : -f * sn;
                                        }
                                    }
                                    v[e] = val * sc;
                                    v[2 + e] = ax == 0 ? der * sc : 0.0f;
                                    v[4 + e] = ax == 1 ? der * sc : 0.0f;
                                    v[6 + e] = ax == 2 ? der * sc : 0.0f;
                                }
                            }
                        }
                        store4(ra_hi, ra_lo, c, v, kSplit);
                    };
                    (void)n_full;
                    // this part's groups g = pt, pt + 3, ... in batches of kPBatch: the batch's TMEM
                    // loads are issued together and waited for once, then its groups are computed as
                    // independent chains; each block is signalled once this part has no more groups in it
                    int next_blk = 0;
                    for (int g0 = pt; g0 < ng; g0 += kPBatch * kPParts) {
                        float buf[kPBatch][8];
#pragma unroll
                        for (int i = 0; i < kPBatch; ++i) {
                            const int c = 8 * (g0 + i * kPParts);
                            if (c < 8 * ng && c < ly.Np) {
                                tmem_ld16x256_x1(th + lq + c, buf[i]);
                                tmem_ld16x256_x1(th + lq16 + c, buf[i] + 4);
                            } else {
#pragma unroll
                                for (int j = 0; j < 8; ++j) buf[i][j] = 0.0f;
                            }
                        }
#pragma unroll
                        for (int i = 0; i < kPBatch; ++i) tmem_wait_ld8(buf[i]);
#pragma unroll
                        for (int i = 0; i < kPBatch; ++i) {
                            const int g = g0 + i * kPParts;
                            if (g < ng) group(8 * g, buf[i]);
                        }
                        const int gl = g0 + kPBatch * kPParts;
                        const int b_next = gl < ng ? gl / 8 : nblk;
                        for (; next_blk < b_next; ++next_blk) block_done(next_blk);
                    }
                    for (; next_blk < nblk; ++next_blk) block_done(next_blk);
                    if (dot) {
                        part += __shfl_xor_sync(0xffffffffu, part, 1);
                        part += __shfl_xor_sync(0xffffffffu, part, 2);
                        if ((lane & 3) == 0) s_f255[pt * kPTile + s] = part;
                    }
                } else if (ly.sdf) {
                    // ---- SDF output layer: f, grad f and the features -> colour input rows ----
                    constexpr int kD = TA::kD;
                    constexpr int Kc = TA::layer(LS).Kp;
                    if (pt == 0) {
                        // column 0 of all 128 rows: f (value rows), then the three gradient rows
                        float c0;
                        tmem_ld32x1(th + lq, c0);
                        tmem_wait_ld();
                        s_g[32 * q + lane] = c0;
                        __syncwarp();
                        if (lane < 8) {
                            const int sm = 8 * q + lane;
                            const float gx = s_g[32 * q + 8 + lane], gy = s_g[32 * q + 16 + lane],
                                        gz = s_g[32 * q + 24 + lane];
                            const float gn = sqrtf(gx * gx + gy * gy + gz * gz);
                            const float inv = gn > 0.0f ? 1.0f / gn : 0.0f;
                            const float* sx = s_x + sm * 8;
                            float* so = s_out + sm * 8;
                            so[0] = p.scale * (c0 + bias[0]);
                            so[1] = gx * sx[3] + gy * sx[4] + gz * sx[5];
                            so[2] = sx[6];
                            so[3] = sx[7];
                            so[4] = gn;
                            so[5] = gx * inv;
                            so[6] = gy * inv;
                            so[7] = gz * inv;
                            // colour prefix: x~, direction encoding, normal (columns 0 .. kD - 1)
                            const uint32_t row = 32 * q + lane;
                            for (int c8 = 0; c8 < kD; c8 += 8) {
                                float o[8];
#pragma unroll
                                for (int jj = 0; jj < 8; ++jj) {
                                    const int col = c8 + jj;
                                    float val = 0.0f;
                                    if (col < 3) val = sx[col];
                                    else if (col < 3 + A::kDirEnc)
                                        val = enc_tab(sx + 3, s_pd + sm * A::kPeDir * 6, A::kPeDir, col - 3, 0);
                                    else if (col < kD + 1) val = so[5 + col - 3 - A::kDirEnc];
                                    o[jj] = val;
                                }
                                st_row8<F16>(A_hi, row, c8, TA::pitch_main(LS), o);
                            }
                        }
                    }
                    if (!epi_sync()) { ok = false; break; }
                    // features: colour group cg = output group cg - kD / 8; column kD holds n_z
                    constexpr int ncg = Kc / 8;
                    const uint32_t rv_hi = smem_u32(A_hi) + a_off(32 * q + (lane & 7), 0, TA::pitch_main(LS));
                    const uint32_t rv_x = smem_u32(X) + a_off(32 * q + (lane & 7), 0, TA::kPitchX > 0 ? TA::kPitchX : 8);
                    for (int b = 0; b * 8 < ncg; ++b) {
                        const int g0 = b * 8 < kD / 8 ? kD / 8 : b * 8;
                        const int gf = g0 + ((pt - g0) % kPParts + kPParts) % kPParts;
                        float d[3][4];
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            const int cg = gf + i * kPParts;
                            const int oc = 8 * (cg - kD / 8);   // first output column of the group
                            if (cg < 8 * b + 8 && cg < ncg && oc < TA::kOutMma) tmem_ld16x256_x1(th + lq + oc, d[i]);
                            else d[i][0] = d[i][1] = d[i][2] = d[i][3] = 0.0f;
                        }
#pragma unroll
                        for (int i = 0; i < 3; ++i) tmem_wait_ld4(d[i]);
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            const int cg = gf + i * kPParts;
                            if (cg >= 8 * b + 8 || cg >= ncg) continue;
                            const int oc = 8 * (cg - kD / 8);
                            float o[2];
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                const int col = oc + fc + e;
                                float val = 0.0f;
                                if (col == 0) val = s_out[s * 8 + 7];
                                else if (col < TA::kOutMma && col < ly.N) val = d[i][e] + bias[col];
                                else if (col < ly.N)
                                    val = s_f255[s] + s_f255[kPTile + s] + s_f255[2 * kPTile + s] + bias[col];
                                o[e] = val;
                            }
                            const int kc = 8 * cg;
                            if (kc < 256) stmatrix1(rv_hi + (uint32_t)(kc >> 3) * 128u, pack2<F16>(o[0], o[1]));
                            else stmatrix1(rv_x + (uint32_t)((kc - 256) >> 3) * 128u, pack2<F16>(o[0], o[1]));
                        }
                        block_done(b);
                    }
                    // the next tile's table (this tile's is no longer read)
                    if (tile + gridDim.x < n_tiles && !build_table(tile + gridDim.x)) { ok = false; break; }
                } else if (L < NL - 1) {
                    // ---- hidden colour layer (ReLU), value rows only ----
                    const int Kn = TA::layer(L + 1).Kp;
                    const uint32_t rv = smem_u32(A_hi) + a_off(32 * q + (lane & 7), 0, Kn);
                    const int ng = Kn / 8;
                    for (int b = 0; b * 8 < ng; ++b) {
                        // this part's (at most three) groups of the block: loads together, one wait
                        const int gf = 8 * b + ((pt - 8 * b) % kPParts + kPParts) % kPParts;
                        float d[3][4];
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            const int c = 8 * (gf + i * kPParts);
                            if (c < 8 * (8 * b + 8) && c < 8 * ng && c < ly.Np) tmem_ld16x256_x1(th + lq + c, d[i]);
                            else d[i][0] = d[i][1] = d[i][2] = d[i][3] = 0.0f;
                        }
#pragma unroll
                        for (int i = 0; i < 3; ++i) tmem_wait_ld4(d[i]);
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            const int g = gf + i * kPParts;
                            if (g >= 8 * b + 8 || g >= ng) continue;
                            const int c = 8 * g;
                            float o[2];
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                const int col = c + fc + e;
                                o[e] = col < ly.N ? fmaxf(d[i][e] + bias[col], 0.0f) : 0.0f;
                            }
                            stmatrix1(rv + (uint32_t)(c >> 3) * 128u, pack2<F16>(o[0], o[1]));
                        }
                        block_done(b);
                    }
                } else {
                    // ---- colour output: the next tile's layer-0 input first (its MMAs run
                    // under this epilogue; every MMA of this tile is complete), then the record ----
                    if (tile + gridDim.x < n_tiles) write_input0();
                    if (pt == 0) {
                        float x0[4];
                        tmem_ld32x4(th + lq, x0);
                        tmem_wait_ld();
                        const int64_t g = tile * kPTile + 8 * q + lane;
                        if (lane < 8 && g < total) {
                            const float* so = s_out + (8 * q + lane) * 8;
                            const float cr = __fdividef(1.0f, 1.0f + __expf(-(x0[0] + bias[0])));
                            const float cgc = __fdividef(1.0f, 1.0f + __expf(-(x0[1] + bias[1])));
                            const float cb = __fdividef(1.0f, 1.0f + __expf(-(x0[2] + bias[2])));
                            float4* R4 = reinterpret_cast<float4*>(p.rec + g);
                            R4[0] = make_float4(so[0], so[1], so[2], so[3]);
                            R4[1] = make_float4(cr, cgc, cb, so[4]);
                            R4[2] = make_float4(so[5], so[6], so[7], 0.0f);
                        }
                    }
                }
                tc_fence_before();
            }
        }
        if (!ok) set_status(p.status, TSDFS_DEV_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kPMmaWarp) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

template <int ARCH, int MODE>
int launch_pipe(const tsdfs_mlp* m, const SampleSource& src, SampleRec* rec, int64_t max_samples, cudaStream_t st) {
    using TA = PipeArch<ARCH>;
    constexpr size_t smem = TA::template smem_bytes<MODE>();
    static_assert(smem <= 232448, "k_mlp_pipe shared memory exceeds 227 KB");
    static int attr_dev[64] = {0};
    int dev = 0, sms = 152;
    int rc = cuda_check(cudaGetDevice(&dev), "mlp_pipe device");
    if (rc) return rc;
    if (dev >= 0 && dev < 64 && !attr_dev[dev]) {
        rc = cuda_check(cudaFuncSetAttribute(k_mlp_pipe<ARCH, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                        "mlp_pipe smem attribute");
        if (rc) return rc;
        attr_dev[dev] = 1;
    }
    PipeParams p{};
    p.packed = static_cast<const uint8_t*>(m->packed);
    p.sdf_w = m->sdf_w;
    p.rgb_w = m->rgb_w;
    for (int a = 0; a < 3; ++a) p.center[a] = m->center[a];
    p.scale = m->scale;
    p.inv_scale = 1.0f / m->scale;
    p.beta = m->beta;
    p.src = src;
    p.rec = rec;
    p.status = device_status_word();
    p.spin = test_spin_limit(kMaxSpin);
    p.withhold = test_withhold_chunk();
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (max_samples + kPTile - 1) / kPTile;
    const unsigned blocks = (unsigned)(tiles < sms ? (tiles < 1 ? 1 : tiles) : sms);
    k_mlp_pipe<ARCH, MODE><<<blocks, PipeMode<MODE>::kThreads, smem, st>>>(p);
    return cuda_check(cudaGetLastError(), "mlp_pipe launch");
}

template <int ARCH>
int launch_pipe_arch(const tsdfs_mlp* m, const SampleSource& src, SampleRec* rec, int64_t max_samples,
                     cudaStream_t st) {
    switch (m->precision) {
        case TSDFS_PREC_F16: return launch_pipe<ARCH, TSDFS_PREC_F16>(m, src, rec, max_samples, st);
        case TSDFS_PREC_BF16: return launch_pipe<ARCH, TSDFS_PREC_BF16>(m, src, rec, max_samples, st);
        case TSDFS_PREC_BF16X2: return launch_pipe<ARCH, TSDFS_PREC_BF16X2>(m, src, rec, max_samples, st);
        default: return fail(TSDFS_E_INVALID, "pipelined network kernel: unsupported precision %d", m->precision);
    }
}

}  // namespace

int launch_mlp_pipe(const tsdfs_mlp* m, const SampleSource& src, SampleRec* rec, int64_t max_samples, cudaStream_t st) {
    if ((reinterpret_cast<uintptr_t>(m->packed) & 15u) != 0) return fail(TSDFS_E_INVALID, "packed weights must be 16-byte aligned");
    if (m->arch == TSDFS_ARCH_TINY) return launch_pipe_arch<TSDFS_ARCH_TINY>(m, src, rec, max_samples, st);
    if (m->arch == TSDFS_ARCH_ROOM) return launch_pipe_arch<TSDFS_ARCH_ROOM>(m, src, rec, max_samples, st);
    return fail(TSDFS_E_UNSUPPORTED, "pipelined network kernel: unknown arch %d", m->arch);
}

}  // namespace tsdfs
