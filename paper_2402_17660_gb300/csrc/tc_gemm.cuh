// Tensor-core GEMM for sm_103a: TMA tile loads into 128B-swizzled shared
// memory, tcgen05.mma issued by one thread with the FP32 accumulator in
// tensor memory (TMEM), and a tcgen05.ld epilogue that applies the same fused
// epilogue functors as the SIMT path.
//
//   C[m][n] = epi( sum_k A[m][k] B[n][k] ),  A [rows][lda], B [rows][ldb},
//   both K-major (row-major with K contiguous).
//
// Two operand modes:
//   BF16   A, B bf16; one kind::f16 MMA per k-step.
//   TF32X3 fp32 A and the weights' TF32 split B = B_hi + B_lo (two fp32
//          arrays of TF32-representable values, see tf32_split); three
//          kind::tf32 MMAs per k-step, A_hi B_hi + A_lo B_hi + A_hi B_lo,
//          within about 3 * 2^-22 |a||b| per product of the fp32 product.
//          A's split is formed in shared memory: two converter warps rewrite
//          each landed A tile into A_hi (in place) and A_lo (a second buffer)
//          at the same byte offsets (an elementwise map, so the 128-byte
//          swizzle carries over), fence it for the async proxy and release
//          the stage to the MMA warp.  No split of an activation ever goes
//          through HBM.
//
// Persistent CTAs walk 128 x BN output tiles.  Warp 0 issues TMA loads into a
// 3-4 stage shared-memory ring (k-blocks of 128-byte rows for BF16, 64-byte
// rows for 3xTF32, whose stage holds four tiles), warp 1 owns TMEM and issues
// the MMAs (32-byte k-steps) into one of two accumulators, so the epilogue of
// a tile overlaps the MMAs of the next.  Sixteen epilogue warps (eight for
// the 128- and 192-wide 3xTF32 tiles) drain TMEM (warp w reads lanes 32*(w%4) .. +31,
// a quarter (half) of the tile's columns each) and run the fused epilogue.  Every mbarrier wait is bounded;
// on expiry the kernel records TNET_ERR_TIMEOUT, the other roles stop, the
// producer waits (bounded) for its own copies in flight, TMEM is freed and
// the kernel returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>
#include <utility>
#include <vector>

#include "internal.cuh"

namespace tnet {
namespace tc {

constexpr int BM = 128, CONV_WARPS = 2;
constexpr int STG_LD = 20;  // floats per staged row (16 + pad, keeps float4 alignment)
constexpr uint32_t kSpinLimit = 1u << 22;

struct TcShape {
    int M[3];                 // rows per class (capacity when rows_dev is set)
    int64_t row0[3];          // first row of each class in A and in the output
    int64_t brow0[3];         // first row of each class's weights in B
    const int32_t *rows_dev;  // optional device row count (class 0), times rows_mul
    int rows_mul;
    int N, K, nclass;
    // testing only (zero in every library call): a smaller bound on each
    // mbarrier wait, and an MMA issuer that issues nothing, so that the
    // bounded waits run out with no MMA and no unconsumed copy in flight
    uint32_t spin_limit;
    int skip_mma;
    // CTAs per thread-block cluster (0 or 1: none; 2 or 4 for a one-class
    // GEMM): the cluster's CTAs take consecutive 128-row tiles of the same
    // column tile, and each loads 1/cl of every B (and B_lo) stage with TMA
    // multicast into all of them, so the weights stream from L2 once per
    // cl * 128 rows instead of once per 128
    int cl;
    // 3xTF32: the operand is SiLU(A) (the converter warps apply silu_f to each
    // landed element before the split), so a layer's activation need not be
    // stored beside its pre-activation
    int a_silu;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// bounded wait on the given phase parity; false when the limit (kSpinLimit
// tries unless `limit` is given) ran out or, when given, the CTA's abort flag
// was raised
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag = nullptr,
                                          uint32_t limit = 0) {
    const uint32_t addr = smem_u32(bar);
    const uint32_t n = limit ? limit : kSpinLimit;
    for (uint32_t it = 0; it < n; ++it) {
        if (abort_flag && (it & 1023u) == 1023u && *abort_flag) return false;
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// the same into every CTA of the cluster in `mask` (same shared-memory offset;
// each destination's barrier at the offset of `bar` receives the bytes)
__device__ __forceinline__ void tma_load_2d_mc(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar,
                                               uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1, "
        "{%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar)), "h"(mask)
        : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// every thread of every CTA of the cluster
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D (TMEM) (+)= A (smem desc) * B (smem desc)^T, kind::f16 with bf16 inputs
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accum)
        : "memory");
}
// the mbarrier arrives once all previously issued MMAs of this thread complete
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// the same arrival on the barrier at this offset in every CTA of `mask`
__device__ __forceinline__ void umma_commit_mc(uint64_t *bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"(mask)
        : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: K-major tile with ROW-byte rows (128 or
// 64) stored in the matching swizzle layout TMA writes; 8-row groups 8 * ROW
// bytes apart.  Swizzle codes: 2 = 128-byte, 4 = 64-byte.
template <int ROW>
__device__ __forceinline__ uint64_t sdesc_sw(uint32_t saddr) {
    static_assert(ROW == 128 || ROW == 64, "row bytes");
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);         // start address / 16
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)((8 * ROW) >> 4) << 32;           // stride byte offset: 8 rows
    d |= (uint64_t)1 << 46;                          // descriptor version for tcgen05
    d |= (uint64_t)(ROW == 128 ? 2 : 4) << 61;       // swizzle mode
    return d;
}

// Instruction descriptor: D f32, A and B bf16 (format 1) or tf32 (format 2),
// both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// D (TMEM) (+)= A * B^T, kind::tf32 (fp32 containers read as TF32)
__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accum)
        : "memory");
}
// The same with A in TMEM: row m of A in lane m, one TF32 element of K per
// 32-bit column (8 columns per k-step)
__device__ __forceinline__ void umma_tf32_at(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                             uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accum)
        : "memory");
}
// this thread's 16 consecutive 32-bit columns of its TMEM lane
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float v[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
        "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
        "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
}

template <int BN, bool X3 = false, bool NK = false>
struct TileCfg {
    // 3xTF32 at BN <= 192 (K beyond two k-blocks): A's split goes to TMEM
    // instead of shared memory.  Four converter warps (one per TMEM lane
    // quadrant) read each landed A row, split it and store A_hi and A_lo with
    // tcgen05.st into a slot of columns after the two accumulators; the MMAs
    // then read only B from shared memory, and the stage needs no A_lo buffer.
    // The narrow tiles (32 or 64 output columns, whose k-blocks carry little
    // MMA work) gain most: their pace is set by splitting A.
    static constexpr bool A_TMEM = X3 && !NK && BN <= 192;
    // one k-block is ROW bytes of K per row: 64 bf16 or 32 fp32 (128-byte
    // rows), or 16 fp32 (64-byte rows) for 3xTF32 with A's split in shared
    // memory, whose stage holds A, A_lo, B and B_lo.  With A in TMEM the
    // 128-byte k-block halves the TMA rows, barrier round trips and loads
    // issued per MMA against 64-byte ones.
    static constexpr int ROW = (X3 && !A_TMEM) ? 64 : 128;
    static constexpr int BKE = ROW / (X3 ? 4 : 2);
    static constexpr int KSTEPS = ROW / 32;  // MMA k-steps (32 bytes of K) per k-block
    static constexpr uint32_t A_BYTES = BM * ROW;
    static constexpr uint32_t B_BYTES = BN * ROW;
    // bytes TMA brings per pipeline stage: A, B (+ B_lo for TF32X3; A_lo is
    // formed in shared memory or TMEM)
    static constexpr uint32_t STAGE_TX = A_BYTES + (X3 ? 2 : 1) * B_BYTES;
    static constexpr int CONV = A_TMEM ? 4 : CONV_WARPS;
    // A_TMEM: slot a holds a k-block's A_hi (ROW / 4 columns) then A_lo at
    // A_COL + a * A_SLOT_COLS; the slots fill TMEM beside the accumulators
    // (2 at BN = 192, 4 at 128) and are released by their own commit barriers
    static constexpr uint32_t A_COL = 2 * BN;
    static constexpr int A_SLOT_COLS = 2 * (ROW / 4);
    static constexpr int A_SLOTS = A_TMEM ? ((512 - 2 * BN) / A_SLOT_COLS > 4 ? 4 : (512 - 2 * BN) / A_SLOT_COLS) : 1;
    static constexpr uint32_t TMEM_COLS =
        A_TMEM ? 512 : (2 * BN <= 64 ? 64 : 2 * BN <= 128 ? 128 : 2 * BN <= 256 ? 256 : 512);
    // epilogue warps: 16, or 8 for the 128- and 192-wide 3xTF32 tiles, whose
    // freed transpose buffers make room for a deeper pipeline; NK (a K of at
    // most two k-blocks, whose epilogue outweighs its MMAs) keeps 16 and 4
    // stages
    static constexpr int EPI = (X3 && !NK && (BN >= 128 || A_TMEM)) ? 8 : 16;
    static constexpr int THREADS = 64 + 32 * (EPI + CONV);
    static constexpr uint32_t STAGE_BYTES = EPI * 32 * STG_LD * 4;  // epilogue transpose buffers
    // 3xTF32: 4 stages, and as many as fit beside the epilogue buffers (6 at
    // BN = 128, 5 at 192, 4 at 256): each stage's split and three MMAs make a
    // long round trip, which the wide radial layers feel.  The narrow tiles (K-wide outputs)
    // keep 4 and a smaller footprint, which leaves room on the SM for the CTAs
    // of the next kernel that programmatic launch brings in early.
    static constexpr int X3_FIT = (int)((232448 - 1024 - 256 - STAGE_BYTES) / (STAGE_TX + A_BYTES));
    // A_TMEM: as many 128-byte stages as fit, at most four (six for the
    // narrow tiles, which stream A).  BF16: four stages (three at BN = 256,
    // where four do not fit beside the epilogue buffers)
    static constexpr int A_FIT = (int)((232448 - 1024 - 256 - STAGE_BYTES) / STAGE_TX);
    static constexpr int A_CAP = BN <= 64 ? 6 : 4;
    static constexpr int STAGES = A_TMEM ? (A_FIT > A_CAP ? A_CAP : A_FIT)
                                         : X3 ? (BN >= 128 && !NK ? (X3_FIT > 6 ? 6 : X3_FIT) : 4)
                                              : (BN >= 256 ? 3 : 4);
    static_assert(!A_TMEM || (A_SLOTS >= 2 && A_COL + A_SLOT_COLS * A_SLOTS <= 512), "A slots exceed TMEM");
    static_assert(STAGES >= 2 && 8 * (3 * STAGES + 5 + A_SLOTS) + 8 <= 256, "pipeline barriers exceed their block");
    static constexpr size_t SMEM =
        1024 + STAGES * (size_t)(STAGE_TX + (X3 && !A_TMEM ? A_BYTES : 0)) + 256 + STAGE_BYTES;
    static_assert(SMEM <= 232448, "dynamic shared memory above 227 KB");
};

// Tile index -> (class, first row, first column); false past the last tile.
// Scalars and selects only: dynamically indexed arrays would live in local memory.
struct TileIter {
    int tilesN, nclass, mt0, mt1, mt2;
    __device__ __forceinline__ bool get(int t, int &z, int &m0, int &n0, int BN_) const {
        const int c0 = mt0 * tilesN, c1 = mt1 * tilesN, c2 = mt2 * tilesN;
        if (t < c0) z = 0;
        else if (nclass > 1 && t < c0 + c1) { z = 1; t -= c0; }
        else if (nclass > 2 && t < c0 + c1 + c2) { z = 2; t -= c0 + c1; }
        else return false;
        m0 = (t / tilesN) * BM;
        n0 = (t % tilesN) * BN_;
        return true;
    }
    // cl > 1 (one class): cluster tile T -> this CTA's tile, rank r of the
    // cluster taking row tile cl * (T / tilesN) + r (past the last row tile
    // its rows are out of range: TMA fills them with zeros and the epilogue
    // stores nothing, but the CTA still loads its share of B for the others)
    __device__ __forceinline__ bool get_cl(int T, int cl, int r, int &m0, int &n0, int BN_) const {
        if (T >= ((mt0 + cl - 1) / cl) * tilesN) return false;
        m0 = ((T / tilesN) * cl + r) * BM;
        n0 = (T % tilesN) * BN_;
        return true;
    }
};
__device__ __forceinline__ int64_t sel3(int z, int64_t a, int64_t b, int64_t c) { return z == 0 ? a : (z == 1 ? b : c); }

template <int BN, class Epi, bool X3, bool NK = false>
__global__ void __launch_bounds__(TileCfg<BN, X3, NK>::THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const __grid_constant__ CUtensorMap tmAlo, const __grid_constant__ CUtensorMap tmBlo, TcShape P,
              Epi epi, int32_t *status) {
    pdl_entry();
    using C = TileCfg<BN, X3, NK>;
    constexpr int STAGES = C::STAGES;
    constexpr int BK = C::BKE;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // stage s: A at sA + s*A_BYTES, B at sB + s*B_BYTES; TF32X3 adds A_lo, B_lo
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * C::A_BYTES;
    uint8_t *sAlo = sB + STAGES * C::B_BYTES;
    uint8_t *sBlo = sAlo + (X3 && !C::A_TMEM ? STAGES * C::A_BYTES : 0);
    uint64_t *full = (uint64_t *)(sBlo + (X3 ? STAGES * C::B_BYTES : 0));
    uint64_t *empty = full + STAGES;
    uint64_t *acc_full = empty + STAGES;
    uint64_t *acc_empty = acc_full + 2;
    uint64_t *conv = acc_empty + 2;  // TF32X3: A_lo of the stage is ready
    uint64_t *drain = conv + STAGES;  // every MMA the issuer started has retired
    uint64_t *aempty = drain + 1;     // A_TMEM: the MMAs that read TMEM A slot a retired
    uint32_t *tmem_slot = (uint32_t *)(aempty + C::A_SLOTS);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    float *stage_all = (float *)((uint8_t *)full + 256);

    // rows per class (class 0 may be bounded by a device-side count)
    int M0 = P.M[0];
    const int M1 = P.nclass > 1 ? P.M[1] : 0, M2 = P.nclass > 2 ? P.M[2] : 0;
    if (P.rows_dev) {
        const int md = *P.rows_dev * P.rows_mul;
        M0 = md < M0 ? md : M0;
    }
    TileIter it;
    it.tilesN = (P.N + BN - 1) / BN;
    it.nclass = P.nclass;
    it.mt0 = (M0 + BM - 1) / BM;
    it.mt1 = (M1 + BM - 1) / BM;
    it.mt2 = (M2 + BM - 1) / BM;
    const int nk = (P.K + BK - 1) / BK;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lim = P.spin_limit;
    // tile walk: over this CTA's tiles, or over its cluster's tiles
    const int cl = P.cl > 1 ? P.cl : 1;
    const int crank = cl > 1 ? (int)cluster_rank() : 0;
    const uint16_t cmask = (uint16_t)((1u << cl) - 1u);
    const int t_first = blockIdx.x / cl, t_step = gridDim.x / cl;
    auto next_tile = [&](int t, int &z, int &m0, int &n0) -> bool {
        if (cl > 1) {
            z = 0;
            return it.get_cl(t, cl, crank, m0, n0, BN);
        }
        return it.get(t, z, m0, n0, BN);
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], cl);  // released by the MMA issuer of every CTA of the cluster
            mbar_init(&conv[s], C::CONV);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], C::EPI);
        }
        mbar_init(drain, 1);
        for (int a = 0; a < C::A_SLOTS; ++a) mbar_init(&aempty[a], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, C::TMEM_COLS);
    fence_before();
    if (cl > 1) cluster_sync();  // every CTA's barriers exist before any multicast reaches them
    else __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            int kg = 0;
            int z, m0, n0;
            for (int t = t_first; next_tile(t, z, m0, n0) && !*abort_flag; t += t_step) {
                for (int kb = 0; kb < nk; ++kb, ++kg) {
                    const int s = kg % STAGES;
                    if (kg >= STAGES && !mbar_wait(&empty[s], ((kg / STAGES) - 1) & 1, abort_flag, lim)) {
                        set_status(status, TNET_ERR_TIMEOUT);
                        *abort_flag = 1;
                        break;
                    }
                    mbar_expect_tx(&full[s], C::STAGE_TX);
                    const int ya = (int)(sel3(z, P.row0[0], P.row0[1], P.row0[2]) + m0);
                    const int yb = (int)(sel3(z, P.brow0[0], P.brow0[1], P.brow0[2]) + n0);
                    tma_load_2d(sA + s * C::A_BYTES, &tmA, kb * BK, ya, &full[s]);
                    if (cl > 1) {  // this CTA's 1/cl of the B rows, into every CTA
                        const int hb = BN / cl;
                        const uint32_t off = (uint32_t)(crank * hb * C::ROW);
                        tma_load_2d_mc(sB + s * C::B_BYTES + off, &tmB, kb * BK, yb + crank * hb, &full[s], cmask);
                        if (X3)
                            tma_load_2d_mc(sBlo + s * C::B_BYTES + off, &tmBlo, kb * BK, yb + crank * hb, &full[s],
                                           cmask);
                    } else {
                        tma_load_2d(sB + s * C::B_BYTES, &tmB, kb * BK, yb, &full[s]);
                        if (X3) tma_load_2d(sBlo + s * C::B_BYTES, &tmBlo, kb * BK, yb, &full[s]);
                    }
                }
            }
            // own copies must land before the CTA exits: a wait that runs out is
            // recorded and taken up again (bounded) on the same barrier
            for (int k = kg > STAGES ? kg - STAGES : 0; k < kg; ++k) {
                bool landed = false;
                for (int r = 0; r < 64 && !landed; ++r) {
                    landed = mbar_wait(&full[k % STAGES], (k / STAGES) & 1, nullptr, lim);
                    if (!landed) set_status(status, TNET_ERR_TIMEOUT);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            const uint32_t idesc = X3 ? idesc_tf32(BM, BN) : idesc_bf16(BM, BN);
            int kg = 0, lt = 0;
            int z, m0, n0;
            for (int t = t_first; !P.skip_mma && next_tile(t, z, m0, n0) && !*abort_flag; t += t_step, ++lt) {
                const int buf = lt & 1;
                if (lt >= 2 && !mbar_wait(&acc_empty[buf], ((lt >> 1) - 1) & 1, abort_flag, lim)) {
                    set_status(status, TNET_ERR_TIMEOUT);
                    *abort_flag = 1;
                    break;
                }
                fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * BN);
                bool ok = true;
                for (int kb = 0; kb < nk; ++kb, ++kg) {
                    const int s = kg % STAGES;
                    if (!mbar_wait(&full[s], (kg / STAGES) & 1, abort_flag, lim) ||
                        (X3 && !mbar_wait(&conv[s], (kg / STAGES) & 1, abort_flag, lim))) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t a0 = smem_u32(sA + s * C::A_BYTES), b0 = smem_u32(sB + s * C::B_BYTES);
                    // 32-byte k-steps: four per 128-byte k-block (bf16), two per
                    // 64-byte k-block (3xTF32)
#pragma unroll
                    for (int k = 0; k < C::KSTEPS; ++k) {
                        const uint64_t da = sdesc_sw<C::ROW>(a0 + k * 32), db = sdesc_sw<C::ROW>(b0 + k * 32);
                        const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
                        if constexpr (C::A_TMEM) {
                            // slot kg mod A_SLOTS: A_hi, then A_lo ROW / 4 columns further
                            const uint32_t ah =
                                tmem + C::A_COL + (uint32_t)(C::A_SLOT_COLS * (kg % C::A_SLOTS) + 8 * k);
                            const uint32_t bl = smem_u32(sBlo + s * C::B_BYTES);
                            umma_tf32_at(d, ah, db, idesc, acc);
                            umma_tf32_at(d, ah + C::ROW / 4, db, idesc, 1u);
                            umma_tf32_at(d, ah, sdesc_sw<C::ROW>(bl + k * 32), idesc, 1u);
                        } else if (X3) {
                            const uint32_t al = smem_u32(sAlo + s * C::A_BYTES), bl = smem_u32(sBlo + s * C::B_BYTES);
                            umma_tf32(d, da, db, idesc, acc);
                            umma_tf32(d, sdesc_sw<C::ROW>(al + k * 32), db, idesc, 1u);
                            umma_tf32(d, da, sdesc_sw<C::ROW>(bl + k * 32), idesc, 1u);
                        } else {
                            umma_bf16(d, da, db, idesc, acc);
                        }
                    }
                    if (cl > 1) umma_commit_mc(&empty[s], cmask);  // the stage is free in every CTA's view
                    else umma_commit(&empty[s]);
                    if constexpr (C::A_TMEM) umma_commit(&aempty[kg % C::A_SLOTS]);
                }
                if (!ok) {
                    set_status(status, TNET_ERR_TIMEOUT);
                    *abort_flag = 1;
                    break;
                }
                umma_commit(&acc_full[buf]);
            }
            // on every path: all MMAs this thread issued retire before the
            // block frees TMEM (a wait that runs out is taken up again)
            umma_commit(drain);
            bool retired = false;
            for (int r = 0; r < 64 && !retired; ++r) {
                retired = mbar_wait(drain, 0, nullptr, lim);
                if (!retired) set_status(status, TNET_ERR_TIMEOUT);
            }
        }
    } else if (warp >= 2 + C::EPI) {
        if (X3) {  // converters: A -> (A_hi, A_lo) for every stage, in k order
            const int ct = threadIdx.x - 32 * (2 + C::EPI);
            int kg = 0;
            bool ok = true;
            int z, m0, n0;
            for (int t = t_first; ok && next_tile(t, z, m0, n0) && !*abort_flag; t += t_step) {
                for (int kb = 0; kb < nk; ++kb, ++kg) {
                    const int s = kg % STAGES;
                    if (!mbar_wait(&full[s], (kg / STAGES) & 1, abort_flag, lim)) {
                        ok = false;
                        break;
                    }
                    if constexpr (C::A_TMEM) {
                        // this lane's row of the tile (= its TMEM lane): 32 fp32
                        // in eight 16-byte chunks, chunk c stored at c ^ (r & 7)
                        // (TMA's 128-byte swizzle)
                        const int q = warp & 3, r = 32 * q + lane;
                        const float4 *row = reinterpret_cast<const float4 *>(sA + s * C::A_BYTES + r * C::ROW);
                        // the slot's last readers, the MMAs of k-block kg - A_SLOTS,
                        // must have retired
                        const int a = kg % C::A_SLOTS;
                        if (kg >= C::A_SLOTS &&
                            !mbar_wait(&aempty[a], ((kg / C::A_SLOTS) - 1) & 1, abort_flag, lim)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        const uint32_t ta =
                            tmem + ((uint32_t)(32 * q) << 16) + C::A_COL + (uint32_t)(C::A_SLOT_COLS * a);
#pragma unroll
                        for (int h16 = 0; h16 < C::ROW / 64; ++h16) {  // 16 elements (four chunks) at a time
                            float h[16], l[16];
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                float4 v = row[(4 * h16 + c) ^ (r & 7)];
                                if (P.a_silu) {
                                    v.x = silu_f(v.x); v.y = silu_f(v.y); v.z = silu_f(v.z); v.w = silu_f(v.w);
                                }
                                tf32_split(v.x, h[4 * c], l[4 * c]);
                                tf32_split(v.y, h[4 * c + 1], l[4 * c + 1]);
                                tf32_split(v.z, h[4 * c + 2], l[4 * c + 2]);
                                tf32_split(v.w, h[4 * c + 3], l[4 * c + 3]);
                            }
                            tmem_st16(ta + 16 * h16, h);
                            tmem_st16(ta + C::ROW / 4 + 16 * h16, l);
                        }
                        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                        fence_before();
                    } else {
                        float4 *hi = reinterpret_cast<float4 *>(sA + s * C::A_BYTES);
                        float4 *lo = reinterpret_cast<float4 *>(sAlo + s * C::A_BYTES);
#pragma unroll 4
                        for (int i = ct; i < (int)(C::A_BYTES / 16); i += 32 * CONV_WARPS) {
                            float4 v = hi[i], l;
                            if (P.a_silu) {
                                v.x = silu_f(v.x); v.y = silu_f(v.y); v.z = silu_f(v.z); v.w = silu_f(v.w);
                            }
                            tf32_split(v.x, v.x, l.x);
                            tf32_split(v.y, v.y, l.y);
                            tf32_split(v.z, v.z, l.z);
                            tf32_split(v.w, v.w, l.w);
                            hi[i] = v;
                            lo[i] = l;
                        }
                        // make the generic-proxy writes visible to the tensor core
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&conv[s]);
                }
            }
            if (!ok) {
                set_status(status, TNET_ERR_TIMEOUT);
                *abort_flag = 1;
            }
        }
    } else {  // epilogue warps 2 .. 2 + C::EPI - 1
        const int q = warp & 3;                  // TMEM lane quadrant this warp may read
        // column slices of at least 16 (one tcgen05.ld.x16); warps past the last
        // slice only take part in the accumulator hand-off
        constexpr int NSLICE = (BN / 16) < (C::EPI / 4) ? (BN / 16) : (C::EPI / 4);
        constexpr int CW = BN / NSLICE;
        const int part = (warp - 2) >> 2;
        const int c_begin = part < NSLICE ? part * CW : 0, c_end = part < NSLICE ? c_begin + CW : 0;
        int lt = 0;
        int z, m0, n0;
        for (int t = t_first; next_tile(t, z, m0, n0) && !*abort_flag; t += t_step, ++lt) {
            const int buf = lt & 1;
            if (!mbar_wait(&acc_full[buf], (lt >> 1) & 1, abort_flag, lim)) {
                set_status(status, TNET_ERR_TIMEOUT);
                *abort_flag = 1;
                break;
            }
            fence_after();
            const int Mrow = (int)sel3(z, M0, M1, M2);
            const int64_t rbase = sel3(z, P.row0[0], P.row0[1], P.row0[2]);
            // TMEM gives thread = row; a shared-memory transpose hands each lane
            // 4 columns of 4 rows instead, so every store instruction of the
            // warp writes 8 rows x 64 contiguous bytes
            float *stg = stage_all + (warp - 2) * 32 * STG_LD;
            const int rsub = lane >> 2, csub = (lane & 3) * 4;
#pragma unroll 1
            for (int c0 = c_begin; c0 < c_end; c0 += 16) {
                const int n = n0 + c0 + csub;
                // the epilogue's loads for this lane's 4 rows first (rows and
                // columns clamped into range), so they overlap the TMEM read
                typename Epi::Pre pr[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int row = m0 + 32 * q + rsub + 8 * k;
                    pr[k] = epi.pre(z, rbase + (row < Mrow ? row : Mrow - 1), n < P.N ? n : P.N - 4);
                }
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * BN + c0), v);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    *reinterpret_cast<float4 *>(stg + lane * STG_LD + 4 * j) =
                        make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                __syncwarp();
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int r = rsub + 8 * k;
                    const int row = m0 + 32 * q + r;
                    const float4 w = *reinterpret_cast<const float4 *>(stg + r * STG_LD + csub);
                    if (row < Mrow && n < P.N) epi.post(z, rbase + row, n, w, pr[k]);
                }
                __syncwarp();
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
        }
    }
    fence_before();
    __syncthreads();
    // no CTA leaves while another may still multicast into its shared memory
    // or release its stages
    if (cl > 1) cluster_sync();
    if (warp == 1) {
        fence_after();
        tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

// ------------------------------------------------------------------ host ---
using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn tensor_map_encoder();  // resolved once through the runtime (tc_gemm.cu)

// 2-D tensor maps (bf16 or fp32): `rows` rows of `cols` elements, row pitch
// `ld` elements, box of `box_rows` x 128 bytes, 128B swizzle, zero fill.
int make_map_bf16(CUtensorMap *m, const void *base, int64_t rows, int64_t cols, int64_t ld, int box_rows);
int make_map_f32(CUtensorMap *m, const void *base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                 int row_bytes);

// Operands of one GEMM: A, B and (TF32X3 only) B's split: B = B_hi, Blo = B_lo.
struct TcOperands {
    const void *A, *B, *Blo;
    int64_t a_rows, lda, b_rows, ldb;
};

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per device and kernel.
// Keyed by the kernel's host-side handle and the device (a template kernel
// used from two translation units can have a handle in each).
inline int ensure_smem_attr(const void *kern, int bytes) {
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> done;  // (kernel handle, device)
    int dev = 0;
    TNET_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> g(mu);
    for (const auto &d : done)
        if (d.first == kern && d.second == dev) return TNET_OK;
    TNET_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    done.emplace_back(kern, dev);
    return TNET_OK;
}

// How many clusters of `cl` CTAs of this kernel the device runs at once (0
// if the query fails); cached per kernel handle, device and cluster size.
inline int max_active_clusters(const void *kern, int threads, int smem, int cl) {
    static std::mutex mu;
    static std::vector<std::pair<std::pair<const void *, int>, int>> done;  // ((kernel, device * 8 + cl), count)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    const int key = dev * 8 + cl;
    std::lock_guard<std::mutex> g(mu);
    for (const auto &d : done)
        if (d.first.first == kern && d.first.second == key) return d.second;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cl, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem;
    cudaLaunchAttribute a[1];
    a[0].id = cudaLaunchAttributeClusterDimension;
    a[0].val.clusterDim.x = (unsigned)cl;
    a[0].val.clusterDim.y = 1;
    a[0].val.clusterDim.z = 1;
    cfg.attrs = a;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        n = 0;
    }
    done.push_back({{kern, key}, n});
    return n;
}

// Launches one persistent GEMM: min(tiles, sms) CTAs, one per SM (`sms` is
// the SM count of the device the stream runs on), in clusters of P.cl when
// the GEMM has one class, the tile splits into cl row groups of whole 8-row
// swizzle atoms, and the device runs such clusters.
template <int BN, bool X3, bool NK = false, class Epi>
int tc_gemm_ops(const TcShape &P0, const TcOperands &o, const Epi &epi, int32_t *status, cudaStream_t st, int sms) {
    using C = TileCfg<BN, X3, NK>;
    TcShape P = P0;
    int cl = P.cl > 1 ? P.cl : 1;
    if (P.nclass != 1 || BN % cl || (BN / cl) % 8) cl = 1;
    const int esz = X3 ? 4 : 2;
    int maxM = 0;
    for (int z = 0; z < P.nclass; ++z) maxM = P.M[z] > maxM ? P.M[z] : maxM;
    if (maxM <= 0 || P.N <= 0) return TNET_OK;
    if (P.N % 4 || (o.lda * esz) % 16 || (o.ldb * esz) % 16 || ((uintptr_t)o.A & 15) || ((uintptr_t)o.B & 15))
        return TNET_ERR_ARG;
    if (X3 && (!o.Blo || ((uintptr_t)o.Blo & 15))) return TNET_ERR_ARG;
    CUtensorMap ma, mb, mal, mbl;
    int rc;
    auto kern = k_tc_gemm<BN, Epi, X3, NK>;
    if ((rc = ensure_smem_attr((const void *)kern, (int)C::SMEM))) return rc;
    if (sms < 1) sms = 1;
    int maxc = 0;
    if (cl > 1) {
        maxc = max_active_clusters((const void *)kern, C::THREADS, (int)C::SMEM, cl);
        if (maxc > sms / cl) maxc = sms / cl;
        if (maxc < 1) cl = 1;
    }
    P.cl = cl;
    const int bbox = BN / cl;  // B rows each CTA loads per stage
    if (X3) {
        if ((rc = make_map_f32(&ma, o.A, o.a_rows, P.K, o.lda, BM, C::ROW))) return rc;
        if ((rc = make_map_f32(&mb, o.B, o.b_rows, P.K, o.ldb, bbox, C::ROW))) return rc;
        if ((rc = make_map_f32(&mbl, o.Blo, o.b_rows, P.K, o.ldb, bbox, C::ROW))) return rc;
        mal = ma;  // unused: A_lo is formed in shared memory or TMEM
    } else {
        if ((rc = make_map_bf16(&ma, o.A, o.a_rows, P.K, o.lda, BM))) return rc;
        if ((rc = make_map_bf16(&mb, o.B, o.b_rows, P.K, o.ldb, bbox))) return rc;
        mal = ma;
        mbl = mb;
    }
    int64_t tiles = 0;
    for (int z = 0; z < P.nclass; ++z) tiles += (int64_t)((P.M[z] + BM - 1) / BM) * ((P.N + BN - 1) / BN);
    int grid;
    if (cl > 1) {  // clusters over cluster tiles (cl row tiles of one column tile)
        const int64_t ctiles = (int64_t)((P.M[0] + BM * cl - 1) / (BM * cl)) * ((P.N + BN - 1) / BN);
        grid = (int)(ctiles < maxc ? ctiles : maxc) * cl;
    } else {
        grid = (int)(tiles < sms ? tiles : sms);
    }
    launch_cluster(kern, grid, C::THREADS, C::SMEM, st, cl, ma, mb, mal, mbl, P, epi, status);
    count_launch();
    TNET_LAUNCH_CHECK();
    return TNET_OK;
}

template <int BN, class Epi>
int tc_gemm(const TcShape &P, const __nv_bfloat16 *A, int64_t a_rows, int64_t lda, const __nv_bfloat16 *B,
            int64_t b_rows, int64_t ldb, const Epi &epi, int32_t *status, cudaStream_t st, int sms) {
    return tc_gemm_ops<BN, false>(P, TcOperands{A, B, nullptr, a_rows, lda, b_rows, ldb}, epi, status, st, sms);
}

inline TcShape tshape(int M, int N, int K) {
    TcShape P{};
    P.M[0] = M;
    P.rows_mul = 1;
    P.N = N;
    P.K = K;
    P.nclass = 1;
    return P;
}

// The three coordinate classes of a node tensor buffer with N atoms (rows
// [0,N), [N,4N), [4N,9N)) against weights stacked [3][F][F].
inline TcShape tshape_classes(int Natoms, int F) {
    TcShape P{};
    P.M[0] = Natoms; P.M[1] = 3 * Natoms; P.M[2] = 5 * Natoms;
    P.row0[0] = 0; P.row0[1] = Natoms; P.row0[2] = 4LL * Natoms;
    P.brow0[0] = 0; P.brow0[1] = F; P.brow0[2] = 2LL * F;
    P.rows_mul = 1;
    P.N = F;
    P.K = F;
    P.nclass = 3;
    return P;
}

}  // namespace tc
}  // namespace tnet
