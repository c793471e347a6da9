// FP16 / BF16 tensor-core (tcgen05) evaluation of the SDF and colour networks.
//
// Tile: 64 samples.  The SDF gradient is carried in forward mode as tangent
// rows.  Two M = 128 accumulators live in tensor memory (TMEM, 2 x 256 fp32
// columns):  acc0 = [value | d/dx] rows, acc1 = [d/dy | d/dz] rows, laid out
// so that TMEM lane quarter q holds samples 16q..16q+15: lanes 0-15 of the
// quarter are the value (acc0) / d/dy (acc1) rows, lanes 16-31 the d/dx (acc0)
// / d/dz (acc1) rows.  Every warp therefore owns 16 value rows, which spreads
// the softplus / sigmoid work over all four SM sub-partitions; hidden layers
// read 16-lane fragments so that one thread holds all four rows of a sample.
// Activations (fp16 / bf16) are the A operands in shared memory, written by
// the epilogue in the no-swizzle K-major core-matrix layout; weights are
// pre-packed in the same layout (tsdfs_pack_mlp) and streamed chunk by chunk
// (kKChunk columns of K) with 1-D bulk TMA copies through a kStages-deep ring.
// The full kernel runs tiles in pairs: the SDF layers of the first tile, then of the second,
// then the colour layers once for both on acc0 (M = 128 rows, all live): the second tile's
// samples in the value-row positions, the first tile's in the d/dx-row positions, which hold
// nothing the colour layers need.  Between the two SDF passes one epilogue thread parks the
// first tile's last SDF input value rows (h, in A0) and its folded colour input extras (in A1)
// in global memory with bulk copies, and brings them back into the d/dx-row groups once the
// second tile's SDF MMAs are done.  The full kernel runs the
// folded tables of tc_common.cuh (TcArch<ARCH, true>): the SDF output layer computes only
// net_0 (N = 16 MMAs on both accumulators, for f and grad f), and the first colour layer
// multiplies the last hidden SDF activation h, still in A0 as that layer's input, by the
// folded weights W_c,feat W_f, with x~, the direction encoding and the unit normal in a
// small block at the start of A1; the 256 feature columns are never formed.
//
// The full kernel (SDF value, gradient and colour): 16 warps, one persistent CTA per SM.
// Warps 0-11 are the epilogue (warp w: TMEM lane quarter w % 4, column part w / 4 of three),
// warp 12 issues the MMAs from precomputed per-chunk records, converged, through one elected
// lane (warp 12 also allocates / frees TMEM), warps 13-15 lane 0
// stream weight chunks, one per slot (two ring stages, and a slot in the free part of A1 while
// the colour layers run): bulk copies issued by one thread towards different mbarriers do not
// overlap (measured), so each slot has a thread of its own.  The value kernel (the
// comparator's coarse pass) has 8 epilogue warps, one MMA warp and one producer warp per ring
// stage.  All hand-offs are mbarriers; every wait is bounded and on timeout the kernel
// records TSDFS_DEV_TIMEOUT, drains its own copies / MMAs and returns.
#include <type_traits>

#include "tc_common.cuh"

namespace tsdfs {

namespace {

// --------------------------------------------------------------------------
// layer tables
// --------------------------------------------------------------------------
constexpr int kTileS = 64;        // samples per tile
constexpr int kStages = 2;        // weight chunks in flight (ring depth), one producer warp each
constexpr uint32_t kBarBytes = 256;  // mbarriers, TMEM slot and abort flag
constexpr int kEpiThreads = 256;  // warps 0-7
constexpr int kMmaWarp = 8;
constexpr int kThreads = 32 * (kMmaWarp + 1 + kStages);
// the full kernel: kEpiWarpsF epilogue warps (kPartsF per TMEM lane quarter, each writing one
// column part of the next operand), then the MMA warp, then one producer warp per stage
constexpr int kEpiWarpsF = 12;
constexpr int kPartsF = kEpiWarpsF / 4;
constexpr int kMmaWarpF = kEpiWarpsF;
// weight slots of the full kernel: the kStages ring stages, and during the colour layers also
// one slot in the A1 operand region (the tangent rows, which the colour layers do not use
// beyond the spill of their input rows), so that more chunks are in flight while the colour
// layers' single-accumulator MMAs consume them; one producer warp per slot
constexpr bool kA1Slots = true;
constexpr int kSlots = kA1Slots ? kStages + 1 : kStages;
constexpr int kThreadsF = 32 * (kMmaWarpF + 1 + kSlots);
constexpr bool kWarpArrive = true;   // one epilogue arrival per warp on the operand / table barriers
constexpr int kEpiArrivals = kWarpArrive ? kEpiWarpsF : 32 * kEpiWarpsF;
static_assert(!kA1Slots || kStages == 2, "the A1 weight slot assumes the 2-stage ring");
constexpr uint32_t kABytes = 64 * 1024;   // one A region (128 rows x 256 bf16)

// the full kernel's own sizes on top of the layer tables
template <int ARCH> struct TcFull : TcArch<ARCH, true> {
    using Base = TcArch<ARCH, true>;
    using Base::layer;
    using Base::kLayers;
    using Base::kXp;
    using Base::stage_bytes;
    using Base::bias_bytes;
    using Base::max_rgb_chunk_bytes;
    using Base::kH;
    using A = Arch<ARCH>;
    // per-tile sample table of the full kernel (coordinates, direction, t, delta, encodings)
    __host__ __device__ static constexpr uint32_t table_bytes() {
        return (uint32_t)(kTileS * (8 + 6 * (A::kPeSdf + A::kPeDir)) * 4);
    }
    // tiles run in pairs: the SDF layers of both tiles, then the colour layers once for both
    __host__ __device__ static constexpr int pair_chunks() { return 2 * Base::sdf_chunks() + Base::rgb_chunks(); }
    __host__ __device__ static constexpr uint32_t pair_chunk_tab_bytes() {
        return (uint32_t)((pair_chunks() * 12 + 15) / 16 * 16);
    }
    // the MMA warp's per-chunk records (descriptors precomputed once per CTA): 32 bytes a chunk
    __host__ __device__ static constexpr uint32_t mma_tab_bytes() { return (uint32_t)pair_chunks() * 32u; }
    __host__ __device__ static constexpr size_t full_smem_bytes() {
        return 2 * (size_t)kABytes + kStages * (size_t)stage_bytes() + bias_bytes() + kBarBytes + table_bytes() +
               pair_chunk_tab_bytes() + mma_tab_bytes();
    }
    // one 8-row core-matrix group of the last SDF layer's input rows (h) and of the folded colour
    // input's extra columns; a pair's first tile parks its value rows (two groups per TMEM lane
    // quarter of each) in global memory while the second tile's SDF layers run
    __host__ __device__ static constexpr uint32_t h_grp() { return (uint32_t)(kH / 8) * 128u; }
    __host__ __device__ static constexpr uint32_t x_grp() { return (uint32_t)(kXp / 8) * 128u; }
    __host__ __device__ static constexpr uint32_t stash_bytes() { return 4u * 2u * (h_grp() + x_grp()); }
    // bytes at the start of A1 holding the folded colour input's x~ / direction / normal
    // columns (128 rows of kXp columns; its h columns are the last SDF layer's input rows in
    // A0), rounded up to 1 KB
    __host__ __device__ static constexpr uint32_t a1_spill() { return (uint32_t)((128 * kXp * 2 + 1023) / 1024 * 1024); }
    // weight slots that fit in the rest of A1 while the colour layers run (at most one)
    __host__ __device__ static constexpr int a1_slots() {
        const int64_t n = ((int64_t)kABytes - a1_spill()) / max_rgb_chunk_bytes();
        return n > 1 ? 1 : (int)n;
    }
};

// one weight chunk of a tile's schedule: its offset and size in the packed weights, the
// weight slot it goes through, its K columns, and whether its slot (an A1 slot after the
// tile's last colour chunk in it) stays with the MMA warp instead of returning to its producer
struct ChunkInfo {
    uint32_t off, bytes;
    uint16_t slot, kc_keep;   // kc_keep: K columns | 0x8000 when the slot is kept
};
static_assert(sizeof(ChunkInfo) == 12, "chunk table entry");

// the MMA warp's record of one weight chunk, written once per CTA: the shared-memory
// descriptors of the chunk's first K step (weights, and the operand rows of both
// accumulators), the instruction descriptor, and the flags below; the issue loop then only
// waits, adds and issues
struct MmaRec {
    uint64_t bd, ad0, ad1;
    uint32_t id, flags;
};
static_assert(sizeof(MmaRec) == 32, "MMA record");
constexpr uint32_t kRecNk = 7u;              // bits 0-2: K steps of 16 columns
constexpr uint32_t kRecTwo = 1u << 3;        // both accumulators (SDF layers)
constexpr uint32_t kRecKeep = 1u << 4;       // the slot stays with the MMA warp (no release)
constexpr uint32_t kRecFirst = 1u << 5;      // first chunk of its layer: wait for the operand
constexpr uint32_t kRecLast = 1u << 6;       // last chunk of its layer: signal the accumulator
constexpr uint32_t kRecRelA1 = 1u << 7;      // after the SDF MMAs: release the A1 slots
constexpr int kRecSlotShift = 8;             // bits 8-9: weight slot
constexpr uint32_t kRecPar = 1u << 10;       // parity of the slot's use within the tile
constexpr uint32_t kRecFlip = 1u << 11;      // the slot's uses per pair of tiles are odd
constexpr uint32_t kRecRestore = 1u << 12;   // first colour chunk: the pair's first tile is back in place

// most CTAs of one launch of the full kernel, and the parking space of each in the caller's
// workspace: the first tile of a pair keeps its last SDF layer's input value rows and its
// folded colour input extras there while the second tile's SDF layers use the operand
// regions (the room networks need the most: 4 x 2 x (4096 + 768) bytes)
constexpr int kPairCtas = 256;
constexpr uint32_t kStashMax = 4u * 2u * (4096u + 768u);

// the value kernel's record of one weight chunk (written once per CTA): packed offset and size
// for its producers; for the MMA warp the descriptors of the chunk's first K step, the
// weights' as if in ring stage 0 (a stage further on adds its offset to the address field)
struct ValRec {
    uint64_t bd0, ad;
    uint32_t id, flags, off, bytes;
};
static_assert(sizeof(ValRec) == 32, "value-kernel record");

struct TcParams {
    const uint8_t* packed;
    const float* sdf_w;
    const float* rgb_w;
    float center[3];
    float inv_scale, scale, beta;
    SampleSource src;
    SampleRec* rec;
    uint8_t* stash;  // the full kernel's parking space: kStashMax bytes per CTA, 16-byte aligned
    uint32_t* status;
    uint32_t spin;   // polls of a bounded wait before it gives up
    int withhold;    // test-only: weight chunk of the first tile whose copy is never issued (-1: none)
};

template <int ARCH, bool F16>
__global__ void __launch_bounds__(kThreadsF, 1) k_mlp_tc(TcParams p) {
    using TA = TcFull<ARCH>;
    using A = Arch<ARCH>;
    constexpr int NL = TA::kLayers;
    constexpr int LS = A::kSdfLayers;
    constexpr uint32_t kStage = TA::stage_bytes();
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* A0 = smem;
    uint8_t* A1 = smem + kABytes;
    uint8_t* stage_base = smem + 2 * kABytes;
    float* sbias = reinterpret_cast<float*>(stage_base + kStages * kStage);
    uint64_t* bars = reinterpret_cast<uint64_t*>(stage_base + kStages * kStage + TA::bias_bytes());
    // bars: full[kSlots], empty[kSlots], acc_ready, a_ready, drain, table, restored (the pair's
    // first tile back in the operand regions)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kSlots + 5);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const uint32_t bar_full0 = smem_u32(bars + 0), bar_empty0 = smem_u32(bars + kSlots);
    const uint32_t bar_acc = smem_u32(bars + 2 * kSlots), bar_a = smem_u32(bars + 2 * kSlots + 1);
    const uint32_t bar_drain = smem_u32(bars + 2 * kSlots + 2), bar_tab = smem_u32(bars + 2 * kSlots + 3);
    const uint32_t bar_rest = smem_u32(bars + 2 * kSlots + 4);
    static_assert(TA::stash_bytes() <= kStashMax, "pair stash size");
    // weight slots: the ring stages, and during the colour layers the free part of A1; a slot's
    // shared address
    constexpr int kColSlots = kA1Slots ? kStages + TA::a1_slots() : kStages;
    static_assert(kColSlots <= kSlots, "weight slot count");
    auto slot_addr = [&](uint32_t sl) -> uint32_t {
        return sl < (uint32_t)kStages ? smem_u32(stage_base + sl * kStage)
                                      : smem_u32(A1) + TA::a1_spill() + (sl - kStages) * (uint32_t)TA::max_rgb_chunk_bytes();
    };
    // per-tile sample table: [x~ (3), direction (3), t, delta] per sample, then sin / cos of the
    // positional encodings of x~ (kPeSdf octaves) and of the direction (kPeDir octaves)
    float* s_x = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(bars) + kBarBytes);
    float* s_pe = s_x + kTileS * 8;
    float* s_pd = s_pe + kTileS * A::kPeSdf * 6;
    ChunkInfo* s_chunks = reinterpret_cast<ChunkInfo*>(reinterpret_cast<uint8_t*>(s_x) + TA::table_bytes());
    MmaRec* s_mma = reinterpret_cast<MmaRec*>(reinterpret_cast<uint8_t*>(s_chunks) + TA::pair_chunk_tab_bytes());
    constexpr int kPC = TA::pair_chunks();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const int64_t total = sample_total(p.src);
    if (total > p.src.capacity) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(p.status, TSDFS_DEV_SAMPLES_OVERFLOW);
        return;
    }
    const int64_t n_tiles = (total + kTileS - 1) / kTileS;
    // pair k: tiles 2k and 2k + 1 (the second past n_tiles when the count is odd: its samples
    // are all invalid, its table zero and its records not written)
    const int64_t n_pairs = (n_tiles + 1) / 2;
    if ((int64_t)blockIdx.x >= n_pairs) return;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kSlots; ++i) {
            mbar_init(bar_full0 + 8 * i, 1);
            mbar_init(bar_empty0 + 8 * i, 1);
        }
        mbar_init(bar_acc, 1);
        mbar_init(bar_a, kEpiArrivals);
        mbar_init(bar_drain, 1);
        mbar_init(bar_tab, kEpiArrivals);
        mbar_init(bar_rest, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // the pair's chunk schedule (the first tile's SDF layers, the second's, then the colour
        // layers once), computed once: SDF chunks alternate over the ring stages, colour chunks
        // cycle over the ring stages and the free part of A1 (the producers and the MMA warp
        // read it instead of re-deriving offsets and slots in their loops)
        static_assert(TA::layer(LS - 1).Np <= 256, "the SDF output layer fits one MMA per accumulator");
        {
            int uses[kSlots];
            for (int i = 0; i < kSlots; ++i) uses[i] = 0;
            const uint32_t a0 = smem_u32(A0), a1 = smem_u32(A1);
            int j = 0, sdf_j = 0, col_j = 0;
            for (int u = 0; u < 2 * LS + (NL - LS); ++u) {
                const int L = u < 2 * LS ? u % LS : u - LS;
                const TcLayer ly = TA::layer(L);
                const uint32_t a_sbo = (uint32_t)(ly.Kp / 8) * 128u;
                for (int c = 0; c < TA::chunks(L); ++c, ++j) {
                    const uint32_t sl = L < LS ? (uint32_t)(sdf_j++ % kStages) : (uint32_t)(col_j % kColSlots);
                    const bool keep = L >= LS && sl >= (uint32_t)kStages && col_j + kColSlots >= TA::rgb_chunks();
                    if (L >= LS) ++col_j;
                    const int kc = TA::chunk_k(L, c);
                    s_chunks[j] = ChunkInfo{(uint32_t)TA::packed_offset(L, c), (uint32_t)TA::chunk_bytes(L, c), (uint16_t)sl,
                                            (uint16_t)(kc | (keep ? 0x8000 : 0))};
                    const int k0 = c * kKChunk;
                    MmaRec r;
                    r.bd = mdesc(slot_addr(sl), 128, (uint32_t)(kc / 8) * 128u);
                    r.ad0 = mdesc(a0 + (uint32_t)(k0 / 8) * 128u, 128, a_sbo);
                    // the folded colour input: its h chunks are the last SDF layer's input rows in
                    // A0 (that layer's layout), its x~ / direction / normal chunk starts A1
                    if (!ly.sdf && ly.idx == 0)
                        r.ad0 = k0 < TA::kH ? mdesc(a0 + (uint32_t)(k0 / 8) * 128u, 128, (TA::kH / 8) * 128u)
                                            : mdesc(a1 + (uint32_t)((k0 - TA::kH) / 8) * 128u, 128, (TA::kXp / 8) * 128u);
                    r.ad1 = mdesc(a1 + (uint32_t)(k0 / 8) * 128u, 128, a_sbo);
                    r.id = idesc_mma<F16>(128, ly.Np);
                    // the A1 slots are released after the second tile's SDF MMAs (the last to read A1)
                    r.flags = (uint32_t)(kc / 16) | (ly.sdf ? kRecTwo : 0u) | (keep ? kRecKeep : 0u) |
                              (c == 0 ? kRecFirst : 0u) | (c + 1 == TA::chunks(L) ? kRecLast : 0u) |
                              (c + 1 == TA::chunks(L) && u == 2 * LS - 1 ? kRecRelA1 : 0u) |
                              (c == 0 && u == 2 * LS ? kRecRestore : 0u) | (sl << kRecSlotShift) |
                              ((uses[sl] & 1) ? kRecPar : 0u);
                    ++uses[sl];
                    s_mma[j] = r;
                }
            }
            for (int jj = 0; jj < kPC; ++jj)
                if (uses[s_chunks[jj].slot] & 1) s_mma[jj].flags |= kRecFlip;
        }
    }
    // all biases of both networks, staged once (the two folded layers' from the packed buffer)
    for (int i = threadIdx.x; i < TA::bias_total(); i += kThreadsF) {
        int L = 0;
        while (L + 1 < NL && TA::bias_offset(L + 1) <= i) ++L;
        const TcLayer ly = TA::layer(L);
        const int j = i - TA::bias_offset(L);
        if (TA::folded(L)) {
            const float* fb = reinterpret_cast<const float*>(p.packed + TA::fold_bias_offset());
            sbias[i] = __ldg(fb + (L == LS ? TA::layer(LS - 1).Np : 0) + j);
        } else {
            const float* W = (ly.sdf ? p.sdf_w : p.rgb_w) + TA::param_offset(L);
            sbias[i] = j < ly.N ? __ldg(W + (int64_t)ly.N * ly.K + j) : 0.0f;
        }
    }
    if (warp == kMmaWarpF) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp > kMmaWarpF) {
        // ------------------ producers: one warp per weight slot (one thread's bulk copies
        // do not overlap each other, and a second spinning lane would stall the first)
        if (lane == 0 && warp - kMmaWarpF - 1 < kColSlots) {
            const uint32_t own = (uint32_t)(warp - kMmaWarpF - 1);
            // ring stages: use u waits for the release of use u - 1; the A1 slot: use u waits
            // for release u (release 0 of a pair is the end of its SDF MMAs, which read A1)
            const uint32_t first = own < (uint32_t)kStages ? 1u : 0u;
            uint32_t issued = 0;
            bool ok = true;
            const uint32_t dst = slot_addr(own);
            for (int64_t pr = blockIdx.x; pr < n_pairs && ok; pr += gridDim.x) {
                for (int j = 0; j < kPC; ++j) {
                    const ChunkInfo ci = s_chunks[j];
                    if (ci.slot != own) continue;
                    // test-only: stop before the withheld chunk of the first pair
                    if (pr == blockIdx.x && j == p.withhold) { ok = false; break; }
                    if (!mbar_wait(bar_empty0 + 8 * own, (issued & 1u) ^ first, abort_flag, p.spin)) { ok = false; break; }
                    mbar_expect_tx(bar_full0 + 8 * own, ci.bytes);
                    bulk_g2s(dst, p.packed + ci.off, ci.bytes, bar_full0 + 8 * own);
                    ++issued;
                }
            }
            if (!ok && issued > 0) {
                // let the copy in flight into this stage land before the CTA exits
                for (uint32_t it = 0; it < kMaxSpin && !mbar_try(bar_full0 + 8 * own, (issued - 1) & 1u); ++it) {
                }
            }
        }
    } else if (warp == kMmaWarpF) {
        // ---------------------------------------------------------- MMA issuer: one record
        // per chunk (descriptors built once per CTA), the next record read while the current
        // chunk's MMAs are issued; the whole warp runs the loop (converged: the descriptors
        // stay warp-uniform) and one elected lane issues the MMAs and commits
        {
            const uint32_t el = elect_one();
            uint32_t lc = 0, tpar = 0;
            bool ok = true;
            for (int64_t pr = blockIdx.x; pr < n_pairs && ok; pr += gridDim.x, tpar ^= 1u) {
                MmaRec cr = s_mma[0];
                for (int j = 0; j < kPC; ++j) {
                    const uint32_t f = cr.flags;
                    if (f & kRecFirst) {
                        if (!__all_sync(0xffffffffu, mbar_wait(bar_a, lc & 1u, abort_flag, p.spin))) { ok = false; break; }
                        // the colour layers' first input rows also hold the pair's first tile, back
                        // from its parking space
                        if ((f & kRecRestore) &&
                            !__all_sync(0xffffffffu, mbar_wait(bar_rest, tpar, abort_flag, p.spin))) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                    }
                    const uint32_t s = (f >> kRecSlotShift) & 3u;
                    const uint32_t ph = ((f & kRecPar) ? 1u : 0u) ^ ((f & kRecFlip) ? tpar : 0u);
                    if (!__all_sync(0xffffffffu, mbar_wait(bar_full0 + 8 * s, ph, abort_flag, p.spin))) { ok = false; break; }
                    tc_fence_after();
                    const MmaRec nx = s_mma[j + 1 < kPC ? j + 1 : 0];
                    const int nk = (int)(f & kRecNk);
                    uint64_t ad0 = cr.ad0, bd = cr.bd;
                    uint32_t acc = (f & kRecFirst) ? 0u : 1u;
                    // each K step of 16 columns moves both operands by two 8x8 core matrices
                    // (256 bytes, 16 in the descriptor's address field, which stays below 2^14
                    // for any shared-memory address), so the loop only adds
                    if (f & kRecTwo) {
                        uint64_t ad1 = cr.ad1;
                        for (int kk = 0; kk < nk; ++kk) {
                            mma_el(el, tmem, ad0, bd, cr.id, acc);
                            mma_el(el, tmem + 256, ad1, bd, cr.id, acc);
                            acc = 1u;
                            ad0 += 16;
                            ad1 += 16;
                            bd += 16;
                        }
                    } else {
                        for (int kk = 0; kk < nk; ++kk) {
                            mma_el(el, tmem, ad0, bd, cr.id, acc);
                            acc = 1u;
                            ad0 += 16;
                            bd += 16;
                        }
                    }
                    // release the slot, except the A1 slot after its last colour chunk of the
                    // tile: the next tile's SDF layers own A1 until their MMAs are done
                    if (!(f & kRecKeep)) commit_el(el, bar_empty0 + 8 * s);
                    if (f & kRecLast) {
                        commit_el(el, bar_acc);
                        ++lc;
                        // the SDF MMAs are the last readers of A1 in this tile: release its slots
                        if (f & kRecRelA1)
                            for (int i = kStages; i < kColSlots; ++i) commit_el(el, bar_empty0 + 8 * i);
                    }
                    cr = nx;
                }
            }
            if (!ok && el) {
                // wait for every MMA issued so far before TMEM is released
                mma_commit(bar_drain);
                for (uint32_t it = 0; it < kMaxSpin && !mbar_try(bar_drain, 0); ++it) {
                }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3, pt = warp >> 2;   // lane quarter, column part
        const bool is_val = lane < 16;
        const int r = 32 * q + lane;                  // TMEM lane / A row of this thread
        const int s = 16 * q + (lane & 15);           // sample within the tile
        const int val_lane = lane & 15;               // lane holding this sample's value row
        const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
        // hidden layers read 16-lane fragments: value rows (acc0) / d/dy rows (acc1) at
        // lanes 32q..32q+15, d/dx (acc0) / d/dz (acc1) at 32q+16..32q+31, so one thread
        // holds all four rows of its samples and applies the slope without a shuffle
        const int fs = lane >> 2, fc = 2 * (lane & 3);
        const uint32_t t_v = tmem + lane_addr, t_x = tmem + (((uint32_t)(32 * q + 16)) << 16);
        const uint32_t t_y = t_v + 256, t_z = t_x + 256;
        const float half_beta = 0.5f * p.beta, inv_beta = 1.0f / p.beta;
        constexpr float kInvSqrt2 = 0.70710678118654752f;
        const SoftplusH2 spk = softplus_h2_consts(half_beta, inv_beta);
        const __half2 inv_sqrt2_h2 = __float2half2_rn(kInvSqrt2);
        // eight encoding columns, entries EN0 .. EN0 + 7 of the SDF input encoding (zero past
        // its end) times scl, one row per thread: A row r is sample s's value row (lanes 0-15)
        // or its d/dx row (lanes 16-31) in A0, its d/dy or d/dz row in A1; EN0 is a
        // compile-time constant, so each column's decode folds away
        auto enc_rows8 = [&](auto en0_tag, int c8, int Kp, float scl) {
            constexpr int EN0 = decltype(en0_tag)::value;
            const float* sx = s_x + s * 8;
            const float* sp = s_pe + s * A::kPeSdf * 6;
            float v0[8], v1[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int en = EN0 + k;
                float val = 0.0f, der = 0.0f;
                int b = -1;
                if (en < 3) {
                    b = en;
                    val = sx[en] * scl;
                    der = scl;
                } else if (en < A::kEnc) {
                    const int qq = en - 3, oct = qq / 6, part = (qq % 6) / 3;
                    b = qq % 3;
                    const float sn = sp[(oct * 3 + b) * 2], cs = sp[(oct * 3 + b) * 2 + 1];
                    const float f = (float)(1 << oct) * scl;
                    val = (part == 0 ? sn : cs) * scl;
                    der = part == 0 ? f * cs : -f * sn;
                }
                v0[k] = is_val ? val : (b == 0 ? der : 0.0f);
                v1[k] = is_val ? (b == 1 ? der : 0.0f) : (b == 2 ? der : 0.0f);
            }
            st_row8<F16>(A0, r, c8, Kp, v0);
            st_row8<F16>(A1, r, c8, Kp, v1);
        };
        uint32_t lc = 0, tab_ph = 0;
        bool ok = true;
        // per-tile sample table (coordinates, direction, t, delta, sin / cos of the encodings):
        // epilogue thread et < 64 looks up sample et, thread et < 192 one (sample, axis)
        const int et = threadIdx.x;
        // the epilogue's arrivals on the operand and table barriers: one per warp once all its
        // lanes are past their writes (and TMEM reads), instead of one per thread
        auto epi_arrive = [&](uint32_t bar) {
            __syncwarp();
            if (!kWarpArrive || lane == 0) mbar_arrive(bar);
        };
        // one epilogue thread parks the pair's first tile (its last SDF layer's input value rows
        // in A0 and its folded colour input extras in A1, two 8-row groups per lane quarter each)
        // in global memory with bulk copies, and brings it back into the tangent-row groups of
        // the same regions once the second tile's SDF MMAs are done
        const bool stasher = et == 4 * 32;
        uint8_t* stash = p.stash + (size_t)blockIdx.x * kStashMax;
        auto build_table = [&](int64_t tile, bool between) -> bool {
                if (between) {
                    // every warp is past the first tile's SDF output layer (the last reader of
                    // its table and the writer of its extras): park the first tile
                    fence_proxy_async();
                    epi_arrive(bar_tab);
                    if (!__all_sync(0xffffffffu, mbar_wait(bar_tab, tab_ph & 1u, abort_flag, p.spin))) return false;
                    ++tab_ph;
                    if (stasher) {
                        for (int qq = 0; qq < 4; ++qq) {
                            bulk_s2g(stash + qq * 2u * TA::h_grp(), smem_u32(A0) + 4u * qq * TA::h_grp(), 2u * TA::h_grp());
                            bulk_s2g(stash + 8u * TA::h_grp() + qq * 2u * TA::x_grp(), smem_u32(A1) + 4u * qq * TA::x_grp(),
                                     2u * TA::x_grp());
                        }
                        bulk_commit();
                    }
                }
                if (et < kTileS) {
                    const int64_t g = tile * kTileS + et;
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
                epi_arrive(bar_tab);
                if (!__all_sync(0xffffffffu, mbar_wait(bar_tab, tab_ph & 1u, abort_flag, p.spin))) return false;
                ++tab_ph;
                // ---- sin / cos of the encodings: thread et < 384 -> (sample et / 6, axis (et / 2) % 3,
                // position or direction encoding et % 2); one sincos at octave 0, then the
                // angle doubled per octave (sin 2x = 2 sin x cos x, cos 2x = (cos x - sin x)
                // (cos x + sin x)): the error grows about twofold per octave, to a few 1e-6
                // at the sixth, far below the FP16 / BF16 rounding of the operands ----
                if (et < 6 * kTileS) {
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
                // the parked rows must have been read before the second tile's layer-0 input
                // overwrites them
                if (between && stasher) bulk_wait_read();
                epi_arrive(bar_tab);
                if (!__all_sync(0xffffffffu, mbar_wait(bar_tab, tab_ph & 1u, abort_flag, p.spin))) return false;
                ++tab_ph;
            return true;
        };
        ok = build_table(2 * (int64_t)blockIdx.x, false);
        for (int64_t pr = blockIdx.x; pr < n_pairs && ok; pr += gridDim.x) {
            // ---- the SDF layers of the pair's two tiles ----
            for (int pass = 0; pass < 2 && ok; ++pass) {
                const int64_t tile = 2 * pr + pass;
                if (pass == 1 && !build_table(tile, true)) {
                    ok = false;
                    break;
                }
                // (the sample table of this tile was built before the loop, during the last
                // pair's colour layers, or just now)
                // ---- layer-0 input: the encoding rows, one row per thread ----
                {
                    constexpr int Kp0 = TA::layer(0).Kp;
                    const int c_lo = part_lo(Kp0, pt, kPartsF), c_hi = part_hi(Kp0, pt, kPartsF);
                    static_for<0, Kp0 / 8>([&](auto g) {
                        constexpr int c8 = 8 * decltype(g)::value;
                        if (c8 >= c_lo && c8 < c_hi) enc_rows8(std::integral_constant<int, c8>{}, c8, Kp0, 1.0f);
                    });
                }
                fence_proxy_async();
                epi_arrive(bar_a);
                int boff = 0;   // this layer's first bias (running, not re-derived)
                for (int L = 0; L < LS; ++L, ++lc) {
                    const TcLayer ly = TA::layer(L);
                    const bool w_ok = mbar_wait(bar_acc, lc & 1u, abort_flag, p.spin);
                    if (!__all_sync(0xffffffffu, w_ok)) { ok = false; break; }
                    tc_fence_after();
                    const float* bias = sbias + boff;
                    boff += ly.Np;
                    if (pass == 1 && L == LS - 1 && stasher) {
                        // the second tile's SDF MMAs are done: bring the first tile back into
                        // the tangent-row groups of A0 and of A1's extras block
                        bulk_wait();
                        mbar_expect_tx(bar_rest, TA::stash_bytes());
                        for (int qq = 0; qq < 4; ++qq) {
                            bulk_g2s(smem_u32(A0) + (4u * qq + 2u) * TA::h_grp(), stash + qq * 2u * TA::h_grp(), 2u * TA::h_grp(),
                                     bar_rest);
                            bulk_g2s(smem_u32(A1) + (4u * qq + 2u) * TA::x_grp(), stash + 8u * TA::h_grp() + qq * 2u * TA::x_grp(),
                                     2u * TA::x_grp(), bar_rest);
                        }
                    }
                    if (ly.sdf && ly.idx < LS - 1) {
                        // ---- hidden SDF layer -> next layer's input (skip concat when due) ----
                        // thread: samples fs, fs + 8 of quarter q; columns c0 + 8g + fc + {0, 1};
                        // stmatrix rows: lane i addresses A row 32q + i (value rows, then d/dx
                        // rows in A0; d/dy, then d/dz in A1), matching the fragment order
                        const int Kn = TA::layer(L + 1).Kp;
                        const float sc = ly.idx + 1 == A::kSkip ? kInvSqrt2 : 1.0f;
                        const uint32_t row0 = smem_u32(A0) + a_off(32 * q + lane, 0, Kn);
                        const uint32_t row1 = smem_u32(A1) + a_off(32 * q + lane, 0, Kn);
                        // the columns below c_fa (whole 16-column blocks of hidden units) are split
                        // among the three parts; the slower tail groups above it (hidden units
                        // < N mixed with the skip input's encoding) go round-robin to the parts
                        const int c_fa = (ly.N / 16) * 16 < Kn ? (ly.N / 16) * 16 : Kn;
                        const int c_lo = part8_lo(c_fa, pt, kPartsF), c_full = part8_hi(c_fa, pt, kPartsF);
                        // 8-column groups, software-pipelined: the TMEM loads of group c + 8 are in
                        // flight while group c is computed.  buf = [value(4) | d/dx(4) | d/dy(4) | d/dz(4)],
                        // each 4 = (sample a, col 0), (a, col 1), (b, col 0), (b, col 1)
                        auto ld8 = [&](int c, float (&d)[16]) {
                            tmem_ld16x256_x1(t_v + c, d);
                            tmem_ld16x256_x1(t_x + c, d + 4);
                            tmem_ld16x256_x1(t_y + c, d + 8);
                            tmem_ld16x256_x1(t_z + c, d + 12);
                        };
                        auto group = [&](int c, const float (&d)[16], auto skip_tag) {
                            constexpr bool kSkipIn = decltype(skip_tag)::value;
                            const float2 b = *reinterpret_cast<const float2*>(bias + c + fc);
                            if constexpr (F16) {
                                // pairs (sample a, columns c, c+1) and (sample b, columns c, c+1)
                                __half2 hv2[2], xv2[2], yv2[2], zv2[2];
    #pragma unroll
                                for (int pr = 0; pr < 2; ++pr) {
                                    __half2 h, sg;
                                    softplus_slope_h2(d[2 * pr] + b.x, d[2 * pr + 1] + b.y, spk, h, sg);
                                    if constexpr (kSkipIn) {
                                        sg = __hmul2(sg, inv_sqrt2_h2);
                                        h = __hmul2(h, inv_sqrt2_h2);
                                    }
                                    hv2[pr] = h;
                                    xv2[pr] = __hmul2(sg, __floats2half2_rn(d[4 + 2 * pr], d[5 + 2 * pr]));
                                    yv2[pr] = __hmul2(sg, __floats2half2_rn(d[8 + 2 * pr], d[9 + 2 * pr]));
                                    zv2[pr] = __hmul2(sg, __floats2half2_rn(d[12 + 2 * pr], d[13 + 2 * pr]));
                                }
                                const uint32_t co = (uint32_t)(c >> 3) * 128u;
                                stmatrix4(row0 + co, h2u(hv2[0]), h2u(hv2[1]), h2u(xv2[0]), h2u(xv2[1]));
                                stmatrix4(row1 + co, h2u(yv2[0]), h2u(yv2[1]), h2u(zv2[0]), h2u(zv2[1]));
                                return;
                            }
                            float hv[4], xv[4], yv[4], zv[4];
    #pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                float h, sg;
                                softplus_slope_tanh(d[e] + ((e & 1) ? b.y : b.x), half_beta, inv_beta, h, sg);
                                if constexpr (kSkipIn) {
                                    sg *= kInvSqrt2;
                                    h *= kInvSqrt2;
                                }
                                hv[e] = h;
                                xv[e] = sg * d[4 + e];
                                yv[e] = sg * d[8 + e];
                                zv[e] = sg * d[12 + e];
                            }
                            const uint32_t co = (uint32_t)(c >> 3) * 128u;
                            stmatrix4(row0 + co, pack2<F16>(hv[0], hv[1]), pack2<F16>(hv[2], hv[3]),
                                      pack2<F16>(xv[0], xv[1]), pack2<F16>(xv[2], xv[3]));
                            stmatrix4(row1 + co, pack2<F16>(yv[0], yv[1]), pack2<F16>(yv[2], yv[3]),
                                      pack2<F16>(zv[0], zv[1]), pack2<F16>(zv[2], zv[3]));
                        };
                        auto body = [&](auto skip_tag) {
                            if (c_full <= c_lo) return;
                            const int ng = (c_full - c_lo) / 8;   // groups of this part below c_full
                            float bufA[16], bufB[16];
                            ld8(c_lo, bufA);
                            tmem_wait_ld16(bufA);
                            int gi = 0;
                            for (; gi + 1 < ng; gi += 2) {
                                const int c0 = c_lo + 8 * gi;
                                ld8(c0 + 8, bufB);
                                group(c0, bufA, skip_tag);
                                tmem_wait_ld16(bufB);
                                const bool more = gi + 2 < ng;
                                if (more) ld8(c0 + 16, bufA);
                                group(c0 + 8, bufB, skip_tag);
                                if (more) tmem_wait_ld16(bufA);
                            }
                            if (gi < ng) group(c_lo + 8 * gi, bufA, skip_tag);   // an odd count: the last group
                        };
                        if (sc != 1.0f) body(std::integral_constant<bool, true>{});
                        else body(std::integral_constant<bool, false>{});
                        // tail: hidden units < N, then gamma(x~) / sqrt(2) (the skip input), then zeros
                        const float* sxa = s_x + (16 * q + fs) * 8;
                        const float* sxb = sxa + 8 * 8;
                        const float* spa = s_pe + (16 * q + fs) * A::kPeSdf * 6;
                        const float* spb = spa + 8 * A::kPeSdf * 6;
                        const int c_tl = Kn < ly.Np ? Kn : ly.Np;   // beyond: encoding columns only
                        for (int c8 = c_fa + 8 * pt; c8 < c_tl; c8 += 8 * kPartsF) {
                            float d[16];   // [value(4) | d/dx(4) | d/dy(4) | d/dz(4)], as ld8
    #pragma unroll
                            for (int j = 0; j < 16; ++j) d[j] = 0.0f;
                            if (c8 < ly.Np) {
                                ld8(c8, d);
                                tmem_wait_ld16(d);
                            }
                            float hv[4], xv[4], yv[4], zv[4];
    #pragma unroll
                            for (int cc = 0; cc < 2; ++cc) {
                                const int col = c8 + fc + cc;
                                if (col < ly.N) {
    #pragma unroll
                                    for (int e = cc; e < 4; e += 2) {
                                        float h, sg;
                                        softplus_slope_tanh(d[e] + bias[col], half_beta, inv_beta, h, sg);
                                        sg *= sc;
                                        hv[e] = h * sc;
                                        xv[e] = sg * d[4 + e];
                                        yv[e] = sg * d[8 + e];
                                        zv[e] = sg * d[12 + e];
                                    }
                                } else {
                                    // encoding entry en of both samples: decoded once per column
                                    const int en = col - ly.N;
                                    const int qq = en - 3, oct = qq / 6, part = (qq % 6) / 3, b = en < 3 ? en : qq % 3;
                                    const bool coord = en < 3, in = en < A::kEnc && (coord || oct < A::kPeSdf);
                                    const float f = coord ? 1.0f : (float)(1 << (oct > 0 ? oct : 0)) * sc;
                                    const int ti = ((coord ? 0 : oct) * 3 + b) * 2;
    #pragma unroll
                                    for (int e = cc; e < 4; e += 2) {
                                        const float* sx = (e & 2) ? sxb : sxa;
                                        const float* sp = (e & 2) ? spb : spa;
                                        float val = 0.0f, der = 0.0f;
                                        if (in) {
                                            if (coord) {
                                                val = sx[b] * sc;
                                                der = sc;
                                            } else {
                                                const float sn = sp[ti], cs = sp[ti + 1];
                                                val = (part == 0 ? sn : cs) * sc;
                                                der = part == 0 ? f * cs : -f * sn;
                                            }
                                        }
                                        hv[e] = val;
                                        xv[e] = b == 0 ? der : 0.0f;
                                        yv[e] = b == 1 ? der : 0.0f;
                                        zv[e] = b == 2 ? der : 0.0f;
                                    }
                                }
                            }
                            const uint32_t co = (uint32_t)(c8 >> 3) * 128u;
                            stmatrix4(row0 + co, pack2<F16>(hv[0], hv[1]), pack2<F16>(hv[2], hv[3]),
                                      pack2<F16>(xv[0], xv[1]), pack2<F16>(xv[2], xv[3]));
                            stmatrix4(row1 + co, pack2<F16>(yv[0], yv[1]), pack2<F16>(yv[2], yv[3]),
                                      pack2<F16>(zv[0], zv[1]), pack2<F16>(zv[2], zv[3]));
                        }
                        // the skip input's 8-column groups past the hidden units' padded width:
                        // gamma(x~) / sqrt(2) only, one row per thread, the same round robin
                        if constexpr (A::kSkip > 0) {
                            if (ly.idx + 1 == A::kSkip) {
                                constexpr int kNs = TA::layer(A::kSkip - 1).N, kNps = TA::layer(A::kSkip - 1).Np;
                                constexpr int kKs = TA::layer(A::kSkip).Kp;
                                constexpr int kFa = (kNs / 16) * 16;
                                static_for<kNps / 8, kKs / 8>([&](auto g) {
                                    constexpr int c8 = 8 * decltype(g)::value;
                                    if (((c8 - kFa) / 8) % kPartsF == pt)
                                        enc_rows8(std::integral_constant<int, c8 - kNs>{}, c8, kKs, kInvSqrt2);
                                });
                            }
                        }
                    } else if (pt == 0) {
                        // ---- SDF output layer, folded to its value column: f and grad f from column 0
                        // of both accumulators; the record's SDF part now, its colour later; the folded
                        // colour input's x~ / direction / normal columns in the value rows at the
                        // start of A1 (its h columns are this layer's input rows in A0) ----
                        constexpr int kDir = A::kDirEnc;
                        constexpr int kXp = TA::kXp;
                        float x0[16], x1[16];
                        tmem_ld16(tmem + lane_addr, x0);
                        tmem_ld16(tmem + 256 + lane_addr, x1);
                        tmem_wait_ld();
                        const float gx = __shfl_sync(0xffffffffu, x0[0], val_lane + 16);
                        const float gz = __shfl_sync(0xffffffffu, x1[0], val_lane + 16);
                        const float gy = x1[0];
                        if (is_val) {
                            float n_hat[3];
                            float venc[kDir];
                            const float f_v = p.scale * (x0[0] + bias[0]);
                            const float gn = sqrtf(gx * gx + gy * gy + gz * gz);
                            const float inv = gn > 0.0f ? 1.0f / gn : 0.0f;
                            n_hat[0] = gx * inv; n_hat[1] = gy * inv; n_hat[2] = gz * inv;
                            const float* ds = s_x + s * 8 + 3;
                            const int64_t g = tile * kTileS + s;
                            if (g < total) {
                                float4* R4 = reinterpret_cast<float4*>(p.rec + g);
                                R4[0] = make_float4(f_v, gx * ds[0] + gy * ds[1] + gz * ds[2], s_x[s * 8 + 6], s_x[s * 8 + 7]);
                                R4[2] = make_float4(n_hat[0], n_hat[1], n_hat[2], 0.0f);
                                reinterpret_cast<float*>(R4 + 1)[3] = gn;
                            }
#pragma unroll
                            for (int e = 0; e < kDir; ++e) venc[e] = enc_tab(ds, s_pd + s * A::kPeDir * 6, A::kPeDir, e, 0);
                            // value rows: [x~ (3), direction encoding, unit normal (3), 0 pad]; the
                            // tangent-row groups are the other tile's (parked, or brought back)
#pragma unroll
                            for (int c0 = 0; c0 < kXp; c0 += 8) {
                                float o[8];
#pragma unroll
                                for (int jj = 0; jj < 8; ++jj) {
                                    const int col = c0 + jj;
                                    float v = 0.0f;
                                    if (col < 3) v = s_x[s * 8 + (col < 3 ? col : 0)];
                                    else if (col < 3 + kDir) v = venc[col - 3 < kDir ? col - 3 : 0];
                                    else if (col < 3 + kDir + 3) v = n_hat[col - 3 - kDir < 3 ? col - 3 - kDir : 0];
                                    o[jj] = v;
                                }
                                st_row8<F16>(A1, r, c0, kXp, o);
                            }
                        }
                    }
                    tc_fence_before();
                    // the first tile's SDF output layer feeds no MMA: the second tile's layer 0 is next
                    if (L < LS - 1 || pass == 1) {
                        fence_proxy_async();
                        epi_arrive(bar_a);
                    }
                }
            }
            if (!ok) break;
            // ---- the colour layers once for both tiles: rows 32q..32q+15 of each lane quarter
            // hold the second tile's samples, rows 32q+16..32q+31 the first's ----
            int boff = TA::bias_offset(LS);
            for (int L = LS; L < NL; ++L, ++lc) {
                const TcLayer ly = TA::layer(L);
                const bool w_ok = mbar_wait(bar_acc, lc & 1u, abort_flag, p.spin);
                if (!__all_sync(0xffffffffu, w_ok)) { ok = false; break; }
                tc_fence_after();
                const float* bias = sbias + boff;
                boff += ly.Np;
                const bool last = L == NL - 1;
                if (!last) {
                    // ---- hidden colour layer (ReLU), all 128 rows, one row per thread (TMEM lane
                    // 32q + lane is operand row 32q + lane): 16 columns a load, the biases read
                    // once per 16 columns for the whole warp ----
                    const int Kn = TA::layer(L + 1).Kp;
                    const int r_own = 32 * q + lane;
                    for (int c0 = part_lo(Kn, pt, kPartsF); c0 < part_hi(Kn, pt, kPartsF); c0 += 16) {
                        float v[16];
                        if (c0 < ly.Np) {
                            tmem_ld16(tmem + lane_addr + c0, v);
                            tmem_wait_ld16(v);
                        } else {
#pragma unroll
                            for (int e = 0; e < 16; ++e) v[e] = 0.0f;
                        }
                        if (c0 + 16 <= ly.N) {
                            // bias in FP32, then round to 16 bits and clamp both halves at once
                            const float4* b4 = reinterpret_cast<const float4*>(bias + c0);
                            uint32_t w[8];
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const float4 b = b4[j];
                                w[2 * j] = relu2<F16>(pack2<F16>(v[4 * j] + b.x, v[4 * j + 1] + b.y));
                                w[2 * j + 1] = relu2<F16>(pack2<F16>(v[4 * j + 2] + b.z, v[4 * j + 3] + b.w));
                            }
                            *reinterpret_cast<uint4*>(A0 + a_off(r_own, c0, Kn)) = make_uint4(w[0], w[1], w[2], w[3]);
                            *reinterpret_cast<uint4*>(A0 + a_off(r_own, c0 + 8, Kn)) = make_uint4(w[4], w[5], w[6], w[7]);
                        } else {
#pragma unroll
                            for (int e = 0; e < 16; ++e) {
                                const int col = c0 + e;
                                v[e] = col < ly.N ? fmaxf(v[e] + bias[col], 0.0f) : 0.0f;
                            }
                            st_row8<F16>(A0, r_own, c0, Kn, v);
                            st_row8<F16>(A0, r_own, c0 + 8, Kn, v + 8);
                        }
                    }
                } else if (pt == 0) {
                    // ---- colour output (sigmoid) -> the records' colour: lane i of quarter q is
                    // sample 16q + i of the second tile (i < 16) or 16q + i - 16 of the first ----
                    float x0[16];
                    tmem_ld16(tmem + lane_addr, x0);
                    tmem_wait_ld();
                    const int64_t g = (2 * pr + (lane < 16 ? 1 : 0)) * kTileS + 16 * q + (lane & 15);
                    if (g < total) {
                        float* R = reinterpret_cast<float*>(p.rec + g);
                        R[4] = __fdividef(1.0f, 1.0f + __expf(-(x0[0] + bias[0])));
                        R[5] = __fdividef(1.0f, 1.0f + __expf(-(x0[1] + bias[1])));
                        R[6] = __fdividef(1.0f, 1.0f + __expf(-(x0[2] + bias[2])));
                    }
                }
                tc_fence_before();
                if (!last) {
                    fence_proxy_async();
                    epi_arrive(bar_a);
                }
                // the next pair's first table, while the colour layers' MMAs run: every warp
                // has left the second tile's SDF output layer (the last reader of its table)
                // once colour layer 0's accumulator is complete
                if (L == LS && pr + gridDim.x < n_pairs && !build_table(2 * (pr + gridDim.x), false)) {
                    ok = false;
                    break;
                }
            }
        }
        if (!ok) set_status(p.status, TSDFS_DEV_TIMEOUT);
        if (stasher) bulk_wait();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarpF) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

// ---- SDF values only (the hierarchical comparator's coarse pass) ----------
// Tile: 128 samples, one value row each (no tangents); one accumulator
// (TMEM columns 0..255); SDF layers only; the output layer needs column 0.
constexpr int kTileV = 128;

template <int ARCH, bool F16>
__global__ void __launch_bounds__(kThreads, 1) k_mlp_tc_value(TcParams p, float* __restrict__ f_out) {
    using TA = TcArch<ARCH>;
    using A = Arch<ARCH>;
    constexpr int LS = A::kSdfLayers;
    constexpr uint32_t kStage = TA::stage_bytes();
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* A0 = smem;
    uint8_t* stage_base = smem + 2 * kABytes;
    float* sbias = reinterpret_cast<float*>(stage_base + kStages * kStage);
    uint64_t* bars = reinterpret_cast<uint64_t*>(stage_base + kStages * kStage + TA::bias_bytes());
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 3);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const uint32_t bar_full0 = smem_u32(bars + 0), bar_empty0 = smem_u32(bars + kStages);
    const uint32_t bar_acc = smem_u32(bars + 2 * kStages), bar_a = smem_u32(bars + 2 * kStages + 1);
    const uint32_t bar_drain = smem_u32(bars + 2 * kStages + 2);
    ValRec* s_rec = reinterpret_cast<ValRec*>(reinterpret_cast<uint8_t*>(bars) + kBarBytes);
    constexpr int kChunksV = TA::sdf_chunks();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t total = sample_total(p.src);
    if (total > p.src.capacity) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(p.status, TSDFS_DEV_SAMPLES_OVERFLOW);
        return;
    }
    const int64_t n_tiles = (total + kTileV - 1) / kTileV;
    if ((int64_t)blockIdx.x >= n_tiles) return;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(bar_full0 + 8 * i, 1);
            mbar_init(bar_empty0 + 8 * i, 1);
        }
        mbar_init(bar_acc, 1);
        mbar_init(bar_a, kEpiThreads);
        mbar_init(bar_drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // per-chunk records (offsets and descriptors computed here once instead of per chunk
        // and tile in the producers' and the MMA warp's loops)
        uint32_t off = 0;
        for (int L = 0, j = 0; L < LS; ++L) {
            const TcLayer ly = TA::layer(L);
            const uint32_t a_sbo = (uint32_t)(ly.Kp / 8) * 128u;
            const int n_mma = L == LS - 1 ? 16 : ly.Np;
            for (int c = 0; c < TA::chunks(L); ++c, ++j) {
                const int kc = TA::chunk_k(L, c);
                const int k0 = c * kKChunk;
                ValRec r;
                r.bd0 = mdesc(smem_u32(stage_base), 128, (uint32_t)(kc / 8) * 128u);
                r.ad = mdesc(smem_u32(A0) + (uint32_t)(k0 / 8) * 128u, 128, a_sbo);
                r.id = idesc_mma<F16>(128, n_mma);
                r.flags = (uint32_t)(kc / 16) | (c == 0 ? kRecFirst : 0u) | (c + 1 == TA::chunks(L) ? kRecLast : 0u);
                r.off = off;
                r.bytes = (uint32_t)TA::chunk_bytes(L, c);
                off += r.bytes;
                s_rec[j] = r;
            }
        }
    }
    for (int i = threadIdx.x; i < TA::bias_offset(LS); i += kThreads) {
        int L = 0;
        while (L + 1 < LS && TA::bias_offset(L + 1) <= i) ++L;
        const TcLayer ly = TA::layer(L);
        const int j = i - TA::bias_offset(L);
        sbias[i] = j < ly.N ? __ldg(p.sdf_w + TA::param_offset(L) + (int64_t)ly.N * ly.K + j) : 0.0f;
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp > kMmaWarp) {
        if (lane == 0) {
            const uint32_t own = (uint32_t)(warp - kMmaWarp - 1);
            uint32_t seq = 0, issued = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
                for (int j = 0; j < kChunksV; ++j, ++seq) {
                    if (seq % kStages != own) continue;
                    if (tile == blockIdx.x && (int)seq == p.withhold) { ok = false; break; }
                    const ValRec& r = s_rec[j];
                    const uint32_t ph = (seq / kStages) & 1u;
                    if (!mbar_wait(bar_empty0 + 8 * own, ph ^ 1u, abort_flag, p.spin)) { ok = false; break; }
                    mbar_expect_tx(bar_full0 + 8 * own, r.bytes);
                    bulk_g2s(smem_u32(stage_base + own * kStage), p.packed + r.off, r.bytes, bar_full0 + 8 * own);
                    ++issued;
                }
            }
            if (!ok && issued > 0) {
                for (uint32_t it = 0; it < kMaxSpin && !mbar_try(bar_full0 + 8 * own, (issued - 1) & 1u); ++it) {
                }
            }
        }
    } else if (warp == kMmaWarp) {
        // the whole warp runs the issue loop (converged: the descriptors stay warp-uniform),
        // one elected lane issues the MMAs and commits
        {
            const uint32_t el = elect_one();
            uint32_t seq = 0, lc = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
                ValRec cr = s_rec[0];
                for (int j = 0; j < kChunksV; ++j, ++seq) {
                    const uint32_t f = cr.flags;
                    if (f & kRecFirst) {
                        if (!__all_sync(0xffffffffu, mbar_wait(bar_a, lc & 1u, abort_flag, p.spin))) { ok = false; break; }
                        tc_fence_after();
                    }
                    const uint32_t s = seq % kStages, ph = (seq / kStages) & 1u;
                    if (!__all_sync(0xffffffffu, mbar_wait(bar_full0 + 8 * s, ph, abort_flag, p.spin))) { ok = false; break; }
                    tc_fence_after();
                    const ValRec nx = s_rec[j + 1 < kChunksV ? j + 1 : 0];
                    // descriptors of the chunk's first K step (the weights' moved to stage s:
                    // kStage / 16 in the address field, which stays below 2^14), advanced by 16
                    // (256 bytes) per K step
                    uint64_t ad = cr.ad, bd = cr.bd0 + (uint64_t)(s * (kStage >> 4));
                    uint32_t acc = (f & kRecFirst) ? 0u : 1u;
                    for (int kk = 0; kk < (int)(f & kRecNk); ++kk) {
                        mma_el(el, tmem, ad, bd, cr.id, acc);
                        acc = 1u;
                        ad += 16;
                        bd += 16;
                    }
                    commit_el(el, bar_empty0 + 8 * s);
                    if (f & kRecLast) {
                        commit_el(el, bar_acc);
                        ++lc;
                    }
                    cr = nx;
                }
            }
            if (!ok && el) {
                mma_commit(bar_drain);
                for (uint32_t it = 0; it < kMaxSpin && !mbar_try(bar_drain, 0); ++it) {
                }
            }
        }
    } else {
        const int q = warp & 3, hf = warp >> 2;
        const int r = 32 * q + lane;  // row = sample within the tile
        const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
        const float half_beta = 0.5f * p.beta, inv_beta = 1.0f / p.beta;
        constexpr float kInvSqrt2 = 0.70710678118654752f;
        uint32_t lc = 0;
        bool ok = true;
        for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
            const int64_t g = tile * kTileV + r;
            const bool valid = g < total;
            int64_t ray = 0;
            float t = 0.0f;
            if (valid) {
                if (p.src.mode == kUniform) {
                    ray = __ldg(p.src.sample_ray + g);
                    const int32_t o0 = __ldg(p.src.offsets + ray), o1 = __ldg(p.src.offsets + ray + 1);
                    const float tn = __ldg(p.src.t_n + ray), tf = __ldg(p.src.t_f + ray);
                    const float dl = (tf - tn) / (float)(o1 - o0);
                    t = tn + ((float)(g - o0) + 0.5f) * dl;
                } else {
                    ray = explicit_ray(p.src, g);
                    t = __ldg(p.src.t + g);
                }
            }
            float xt[3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                xt[a] = (__ldg(p.src.ray_o + 3 * ray + a) + t * __ldg(p.src.ray_d + 3 * ray + a) - p.center[a]) * p.inv_scale;
            {
                constexpr int Kp0 = TA::layer(0).Kp;
                for (int k0 = hf * (Kp0 / 2); k0 < (hf + 1) * (Kp0 / 2); k0 += 8) {
                    float v0[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) v0[j] = k0 + j < A::kEnc ? enc_val(xt, k0 + j, A::kPeSdf, 0, false) : 0.0f;
                    st_row8<F16>(A0, r, k0, Kp0, v0);
                }
            }
            fence_proxy_async();
            mbar_arrive(bar_a);
            int boff = 0;
            for (int L = 0; L < LS; ++L, ++lc) {
                const TcLayer ly = TA::layer(L);
                const bool w_ok = mbar_wait(bar_acc, lc & 1u, abort_flag, p.spin);
                if (!__all_sync(0xffffffffu, w_ok)) { ok = false; break; }
                tc_fence_after();
                const float* bias = sbias + boff;
                boff += ly.Np;
                if (L < LS - 1) {
                    const int Kn = TA::layer(L + 1).Kp;
                    const float sc = ly.idx + 1 == A::kSkip ? kInvSqrt2 : 1.0f;
                    for (int c0 = half_lo(Kn, hf); c0 < half_hi(Kn, hf); c0 += 16) {
                        float x0[16], o[16];
                        if (c0 < ly.Np) {
                            tmem_ld16(tmem + lane_addr + c0, x0);
                            tmem_wait_ld();
                        }
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int col = c0 + j;
                            if (col < ly.N) {
                                float h, sg;
                                softplus_slope_tanh(x0[j] + bias[col], half_beta, inv_beta, h, sg);
                                o[j] = h * sc;
                            } else {
                                const int e = col - ly.N;
                                o[j] = e < A::kEnc ? enc_val(xt, e, A::kPeSdf, 0, false) * sc : 0.0f;
                            }
                        }
                        st_row8<F16>(A0, r, c0, Kn, o);
                        st_row8<F16>(A0, r, c0 + 8, Kn, o + 8);
                    }
                } else if (hf == 0) {
                    float x0[16];
                    tmem_ld16(tmem + lane_addr, x0);
                    tmem_wait_ld();
                    if (valid) f_out[g] = p.scale * (x0[0] + bias[0]);
                }
                tc_fence_before();
                if (L < LS - 1) {
                    fence_proxy_async();
                    mbar_arrive(bar_a);
                }
            }
        }
        if (!ok) set_status(p.status, TSDFS_DEV_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
    }
}

template <int ARCH, bool F16>
int launch_tc_value(const tsdfs_mlp* m, const SampleSource& src, float* f_out, cudaStream_t st) {
    using TA = TcArch<ARCH>;
    const size_t smem = 2 * kABytes + kStages * (size_t)TA::stage_bytes() + TA::bias_bytes() + kBarBytes +
                        (size_t)TA::sdf_chunks() * sizeof(ValRec);
    static bool attr[2] = {false, false};
    if (!attr[ARCH]) {
        int rc = cuda_check(cudaFuncSetAttribute(k_mlp_tc_value<ARCH, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem),
                            "mlp_tc_value smem attribute");
        if (rc) return rc;
        attr[ARCH] = true;
    }
    TcParams p{};
    p.packed = static_cast<const uint8_t*>(m->packed);
    p.sdf_w = m->sdf_w;
    p.rgb_w = m->rgb_w;
    for (int a = 0; a < 3; ++a) p.center[a] = m->center[a];
    p.scale = m->scale;
    p.inv_scale = 1.0f / m->scale;
    p.beta = m->beta;
    p.src = src;
    p.status = device_status_word();
    p.spin = test_spin_limit(kMaxSpin);
    p.withhold = test_withhold_chunk();
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (src.mode == kUniform && !src.sample_ray) return fail(TSDFS_E_INVALID, "value pass needs the sample ray index");
    const int64_t tiles = (sample_bound(src) + kTileV - 1) / kTileV;
    const unsigned blocks = (unsigned)(tiles < sms ? (tiles < 1 ? 1 : tiles) : sms);
    k_mlp_tc_value<ARCH, F16><<<blocks, kThreads, smem, st>>>(p, f_out);
    return cuda_check(cudaGetLastError(), "mlp_tc_value launch");
}

// ---- pack fp32 [N][K] weights into the bf16 chunked core-matrix layout ----
template <int ARCH, bool F16>
__global__ void k_pack(const float* __restrict__ sdf_w, const float* __restrict__ rgb_w, uint16_t* __restrict__ out,
                       uint32_t* status) {
    using TA = TcArch<ARCH>;
    const int64_t total = TA::packed_bytes() / 2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        // locate the (layer, chunk) holding element e
        int L = 0, c = 0;
        int64_t base = 0;
        bool found = false;
        for (int l = 0; l < TA::kLayers && !found; ++l)
            for (int cc = 0; cc < TA::chunks(l); ++cc) {
                const int64_t n = TA::chunk_bytes(l, cc) / 2;
                if (e < base + n) { L = l; c = cc; found = true; break; }
                base += n;
            }
        const TcLayer ly = TA::layer(L);
        const int kc = TA::chunk_k(L, c);
        const int64_t w = e - base;
        const int core = (int)(w / 64), within = (int)(w % 64);
        const int n = (core / (kc / 8)) * 8 + within / 8;
        const int k = c * kKChunk + (core % (kc / 8)) * 8 + within % 8;
        const float* W = (ly.sdf ? sdf_w : rgb_w) + TA::param_offset(L);
        const float v = (n < ly.N && k < ly.K) ? W[(int64_t)n * ly.K + k] : 0.0f;
        if (!isfinite(v)) set_status(status, TSDFS_DEV_NONFINITE);
        if constexpr (F16) {
            __half h = __float2half_rn(v);
            out[e] = *reinterpret_cast<uint16_t*>(&h);
        } else {
            __nv_bfloat16 h = __float2bfloat16_rn(v);
            out[e] = *reinterpret_cast<uint16_t*>(&h);
        }
    }
}

// ---- the serial kernel's folded layers: the SDF output layer's value row, and the first
// colour layer on [h, x~, direction, normal] with W_c,feat W_f (FP32 sums, then rounded like
// every packed weight) and the FP32 biases of both ----
template <int ARCH, bool F16>
__global__ void k_pack_fold(const float* __restrict__ sdf_w, const float* __restrict__ rgb_w, uint8_t* __restrict__ out,
                            uint32_t* status) {
    using TF = TcArch<ARCH, true>;
    using A = Arch<ARCH>;
    constexpr int LS = A::kSdfLayers;
    constexpr Layer lo = A::sdf(LS - 1), c0 = A::rgb(0);
    const float* Wo = sdf_w + sdf_layer_offset<ARCH>(LS - 1);   // [1 + feat][kH], then its bias
    const float* bo = Wo + (int64_t)lo.out * lo.in;
    const float* Wc = rgb_w + rgb_layer_offset<ARCH>(0);         // [out][kX + feat], then its bias
    const float* bc = Wc + (int64_t)c0.out * c0.in;
    constexpr int kFeat = A::kFeat;
    const int64_t base = TF::packed_offset(LS - 1, 0);
    const int64_t n_w = (TF::layer_bytes(LS - 1) + TF::layer_bytes(LS)) / 2;
    const int64_t n_b = TF::fold_bias_count();
    uint16_t* out16 = reinterpret_cast<uint16_t*>(out + base);
    float* fb = reinterpret_cast<float*>(out + TF::fold_bias_offset());
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_w + n_b; e += (int64_t)gridDim.x * blockDim.x) {
        if (e >= n_w) {
            // biases: the value column's, then the folded colour layer's
            const int i = (int)(e - n_w);
            float v = 0.0f;
            if (i < TF::layer(LS - 1).Np) {
                v = i == 0 ? bo[0] : 0.0f;
            } else {
                const int n = i - TF::layer(LS - 1).Np;
                if (n < c0.out) {
                    float acc = bc[n];
                    for (int j = 0; j < kFeat; ++j) acc = fmaf(Wc[(int64_t)n * c0.in + TF::kX + j], bo[1 + j], acc);
                    v = acc;
                }
            }
            if (!isfinite(v)) set_status(status, TSDFS_DEV_NONFINITE);
            fb[i] = v;
            continue;
        }
        // locate the layer and chunk holding element e of the folded weights
        const int L = e < TF::layer_bytes(LS - 1) / 2 ? LS - 1 : LS;
        int64_t w = L == LS - 1 ? e : e - TF::layer_bytes(LS - 1) / 2;
        int c = 0;
        while (c + 1 < TF::chunks(L) && w >= TF::chunk_bytes(L, c) / 2) {
            w -= TF::chunk_bytes(L, c) / 2;
            ++c;
        }
        const int kc = TF::chunk_k(L, c);
        const int core = (int)(w / 64), within = (int)(w % 64);
        const int n = (core / (kc / 8)) * 8 + within / 8;
        const int k = c * kKChunk + (core % (kc / 8)) * 8 + within % 8;
        float v = 0.0f;
        if (L == LS - 1) {
            if (n == 0 && k < lo.in) v = Wo[k];
        } else if (n < c0.out) {
            if (k < TF::kH) {
                float acc = 0.0f;
                for (int j = 0; j < kFeat; ++j)
                    acc = fmaf(Wc[(int64_t)n * c0.in + TF::kX + j], Wo[(int64_t)(1 + j) * lo.in + k], acc);
                v = acc;
            } else if (k - TF::kH < TF::kX) {
                v = Wc[(int64_t)n * c0.in + (k - TF::kH)];
            }
        }
        if (!isfinite(v)) set_status(status, TSDFS_DEV_NONFINITE);
        if constexpr (F16) {
            __half h = __float2half_rn(v);
            out16[e] = *reinterpret_cast<uint16_t*>(&h);
        } else {
            __nv_bfloat16 h = __float2bfloat16_rn(v);
            out16[e] = *reinterpret_cast<uint16_t*>(&h);
        }
    }
}

template <int ARCH, bool F16>
int launch_tc(const tsdfs_mlp* m, const SampleSource& src, SampleRec* rec, int64_t max_samples, uint8_t* stash,
              cudaStream_t st) {
    using TA = TcFull<ARCH>;
    constexpr size_t smem = TA::full_smem_bytes();
    static_assert(smem <= 232448, "k_mlp_tc shared memory exceeds 227 KB");
    static bool attr[2] = {false, false};
    if (!attr[ARCH]) {
        int rc = cuda_check(cudaFuncSetAttribute(k_mlp_tc<ARCH, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                            "mlp_tc smem attribute");
        if (rc) return rc;
        attr[ARCH] = true;
    }
    TcParams p{};
    p.packed = static_cast<const uint8_t*>(m->packed);
    p.sdf_w = m->sdf_w;
    p.rgb_w = m->rgb_w;
    for (int a = 0; a < 3; ++a) p.center[a] = m->center[a];
    p.scale = m->scale;
    p.inv_scale = 1.0f / m->scale;
    p.beta = m->beta;
    p.src = src;
    p.rec = rec;
    p.stash = stash;
    p.status = device_status_word();
    p.spin = test_spin_limit(kMaxSpin);
    p.withhold = test_withhold_chunk();
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t pairs = ((max_samples + kTileS - 1) / kTileS + 1) / 2;
    int64_t blocks = pairs < sms ? pairs : sms;
    if (blocks > kPairCtas) blocks = kPairCtas;
    if (blocks < 1) blocks = 1;
    k_mlp_tc<ARCH, F16><<<(unsigned)blocks, kThreadsF, smem, st>>>(p);
    return cuda_check(cudaGetLastError(), "mlp_tc launch");
}

}  // namespace

int mlp_tc_available(int arch) { return arch == TSDFS_ARCH_TINY || arch == TSDFS_ARCH_ROOM; }

size_t mlp_tc_stash_bytes() { return (size_t)kPairCtas * kStashMax; }

int launch_mlp_full_tc(const tsdfs_mlp* m, const SampleSource& src, SampleRec* rec, int64_t max_samples,
                       uint8_t* stash, cudaStream_t st) {
    if ((reinterpret_cast<uintptr_t>(m->packed) & 15u) != 0) return fail(TSDFS_E_INVALID, "packed weights must be 16-byte aligned");
    if (!stash || (reinterpret_cast<uintptr_t>(stash) & 15u) != 0)
        return fail(TSDFS_E_INVALID, "the network kernel's parking space must be 16-byte aligned workspace");
    const bool f16 = m->precision == TSDFS_PREC_F16;
    if (m->arch == TSDFS_ARCH_TINY)
        return f16 ? launch_tc<TSDFS_ARCH_TINY, true>(m, src, rec, max_samples, stash, st)
                   : launch_tc<TSDFS_ARCH_TINY, false>(m, src, rec, max_samples, stash, st);
    return f16 ? launch_tc<TSDFS_ARCH_ROOM, true>(m, src, rec, max_samples, stash, st)
               : launch_tc<TSDFS_ARCH_ROOM, false>(m, src, rec, max_samples, stash, st);
}

int launch_mlp_value_tc(const tsdfs_mlp* m, const SampleSource& src, float* f_out, cudaStream_t st) {
    const bool f16 = m->precision == TSDFS_PREC_F16;
    if (m->arch == TSDFS_ARCH_TINY)
        return f16 ? launch_tc_value<TSDFS_ARCH_TINY, true>(m, src, f_out, st)
                   : launch_tc_value<TSDFS_ARCH_TINY, false>(m, src, f_out, st);
    return f16 ? launch_tc_value<TSDFS_ARCH_ROOM, true>(m, src, f_out, st)
               : launch_tc_value<TSDFS_ARCH_ROOM, false>(m, src, f_out, st);
}

// the whole packed buffer: the unfolded layers (read by every tensor-core kernel), then the
// serial kernel's folded layers and their biases
int64_t packed_bytes(int arch) {
    return arch == TSDFS_ARCH_TINY ? TcArch<TSDFS_ARCH_TINY, true>::packed_bytes()
                                   : (arch == TSDFS_ARCH_ROOM ? TcArch<TSDFS_ARCH_ROOM, true>::packed_bytes() : 0);
}

}  // namespace tsdfs

using namespace tsdfs;

extern "C" size_t tsdfs_packed_size(int32_t arch) { return (size_t)packed_bytes(arch); }

extern "C" int tsdfs_pack_mlp(const tsdfs_mlp* m, void* packed, tsdfs_stream_t stream) {
    if (!m || !packed || !m->sdf_w || !m->rgb_w) return fail(TSDFS_E_INVALID, "mlp, its weights and packed must be non-NULL");
    if (m->arch != TSDFS_ARCH_TINY && m->arch != TSDFS_ARCH_ROOM) return fail(TSDFS_E_INVALID, "unknown arch %d", m->arch);
    if ((reinterpret_cast<uintptr_t>(packed) & 15u) != 0) return fail(TSDFS_E_INVALID, "packed must be 16-byte aligned");
    const bool tiny = m->arch == TSDFS_ARCH_TINY;
    const int64_t plain = tiny ? TcArch<TSDFS_ARCH_TINY>::packed_bytes() : TcArch<TSDFS_ARCH_ROOM>::packed_bytes();
    const int64_t n = plain / 2, nf = (packed_bytes(m->arch) - plain) / 2;
    cudaStream_t st = (cudaStream_t)stream;
    ProfScope ps("pack", st);
    uint16_t* out = static_cast<uint16_t*>(packed);
    uint8_t* out8 = static_cast<uint8_t*>(packed);
    uint32_t* dsw = device_status_word();
    const bool f16 = m->precision == TSDFS_PREC_F16;
    if (tiny) {
        if (f16) {
            k_pack<TSDFS_ARCH_TINY, true><<<grid_1d(n, 256), 256, 0, st>>>(m->sdf_w, m->rgb_w, out, dsw);
            k_pack_fold<TSDFS_ARCH_TINY, true><<<grid_1d(nf, 256), 256, 0, st>>>(m->sdf_w, m->rgb_w, out8, dsw);
        } else {
            k_pack<TSDFS_ARCH_TINY, false><<<grid_1d(n, 256), 256, 0, st>>>(m->sdf_w, m->rgb_w, out, dsw);
            k_pack_fold<TSDFS_ARCH_TINY, false><<<grid_1d(nf, 256), 256, 0, st>>>(m->sdf_w, m->rgb_w, out8, dsw);
        }
    } else {
        if (f16) {
            k_pack<TSDFS_ARCH_ROOM, true><<<grid_1d(n, 256), 256, 0, st>>>(m->sdf_w, m->rgb_w, out, dsw);
            k_pack_fold<TSDFS_ARCH_ROOM, true><<<grid_1d(nf, 256), 256, 0, st>>>(m->sdf_w, m->rgb_w, out8, dsw);
        } else {
            k_pack<TSDFS_ARCH_ROOM, false><<<grid_1d(n, 256), 256, 0, st>>>(m->sdf_w, m->rgb_w, out, dsw);
            k_pack_fold<TSDFS_ARCH_ROOM, false><<<grid_1d(nf, 256), 256, 0, st>>>(m->sdf_w, m->rgb_w, out8, dsw);
        }
    }
    return cuda_check(cudaGetLastError(), "tsdfs_pack_mlp launch");
}

namespace tsdfs {
namespace {
__global__ void k_check_finite(const float* __restrict__ w, int64_t n, uint32_t* status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(__ldg(w + i))) {
            set_status(status, TSDFS_DEV_NONFINITE);
            return;
        }
}
}  // namespace
}  // namespace tsdfs

extern "C" int tsdfs_check_mlp(const tsdfs_mlp* m, tsdfs_stream_t stream) {
    if (!m || !m->sdf_w || !m->rgb_w) return fail(TSDFS_E_INVALID, "mlp and its weights must be non-NULL");
    if (m->arch != TSDFS_ARCH_TINY && m->arch != TSDFS_ARCH_ROOM) return fail(TSDFS_E_INVALID, "unknown arch %d", m->arch);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t ns = m->arch == TSDFS_ARCH_TINY ? sdf_param_count<TSDFS_ARCH_TINY>() : sdf_param_count<TSDFS_ARCH_ROOM>();
    const int64_t nr = m->arch == TSDFS_ARCH_TINY ? rgb_param_count<TSDFS_ARCH_TINY>() : rgb_param_count<TSDFS_ARCH_ROOM>();
    ProfScope ps("check_mlp", st);
    k_check_finite<<<grid_1d(ns, 256), 256, 0, st>>>(m->sdf_w, ns, device_status_word());
    k_check_finite<<<grid_1d(nr, 256), 256, 0, st>>>(m->rgb_w, nr, device_status_word());
    return cuda_check(cudaGetLastError(), "tsdfs_check_mlp launch");
}
