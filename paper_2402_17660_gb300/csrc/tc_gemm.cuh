// BF16 tensor-core GEMM for sm_103a: TMA tile loads into 128B-swizzled
// shared memory, tcgen05.mma issued by one thread with the FP32 accumulator
// in tensor memory (TMEM), and a tcgen05.ld epilogue that applies the same
// fused epilogue functors as the SIMT path.
//
//   C[m][n] = epi( sum_k A[m][k] B[n][k] ),  A [rows][lda], B [rows][ldb] bf16,
//   both K-major (row-major with K contiguous).
//
// One CTA computes one 128 x BN output tile.  Warp 0 issues TMA loads into a
// 4-stage ring, warp 1 owns TMEM and issues the MMAs (K = 16 per instruction,
// four per 64-wide k-block), warps 2..5 drain TMEM (warp w reads lanes
// 32*(w%4) .. +31) and run the epilogue.  Every mbarrier wait is bounded; on
// expiry the kernel records TNET_ERR_TIMEOUT, waits (bounded) for its own
// copies in flight, frees TMEM and returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "internal.cuh"

namespace tnet {
namespace tc {

constexpr int BM = 128, BK = 64, STAGES = 4, THREADS = 192;
constexpr uint32_t kSpinLimit = 1u << 22;

struct TcShape {
    int M[3];                 // rows per class (capacity when rows_dev is set)
    int64_t row0[3];          // first row of each class in A and in the output
    int64_t brow0[3];         // first row of each class's weights in B
    const int32_t *rows_dev;  // optional device row count (class 0), times rows_mul
    int rows_mul;
    int N, K, nclass;
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
// bounded wait on the given phase parity; false when the limit ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t addr = smem_u32(bar);
    for (uint32_t it = 0; it < kSpinLimit; ++it) {
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

// Shared-memory matrix descriptor: K-major tile with 128-byte rows stored in
// the 128B-swizzle layout TMA writes; 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);  // start address / 16
    d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                   // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                   // 128-byte swizzle
    return d;
}

// Instruction descriptor: D f32, A and B bf16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int BN>
struct TileCfg {
    static constexpr uint32_t A_BYTES = BM * BK * 2;
    static constexpr uint32_t B_BYTES = BN * BK * 2;
    static constexpr uint32_t TMEM_COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
    static constexpr size_t SMEM = 1024 + STAGES * (size_t)(A_BYTES + B_BYTES) + 256;
};

template <int BN, class Epi>
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcShape P, Epi epi,
              int32_t *status) {
    using C = TileCfg<BN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * C::A_BYTES;
    uint64_t *full = (uint64_t *)(sB + STAGES * C::B_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *done = empty + STAGES;
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int z = blockIdx.z;
    int M = P.M[z];
    if (z == 0 && P.rows_dev) {
        const int md = *P.rows_dev * P.rows_mul;
        M = md < M ? md : M;
    }
    const int m0 = blockIdx.x * BM;
    if (m0 >= M) return;  // whole CTA leaves before touching TMEM
    const int n0 = blockIdx.y * BN;
    const int nk = (P.K + BK - 1) / BK;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, C::TMEM_COLS);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            int issued = 0;
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % STAGES;
                if (kb >= STAGES && !mbar_wait(&empty[s], ((kb / STAGES) - 1) & 1)) {
                    set_status(status, TNET_ERR_TIMEOUT);
                    *abort_flag = 1;
                    break;
                }
                mbar_expect_tx(&full[s], C::A_BYTES + C::B_BYTES);
                tma_load_2d(sA + s * C::A_BYTES, &tmA, kb * BK, (int)(P.row0[z] + m0), &full[s]);
                tma_load_2d(sB + s * C::B_BYTES, &tmB, kb * BK, (int)(P.brow0[z] + n0), &full[s]);
                issued = kb + 1;
            }
            for (int kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
                mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1);  // own copies have landed
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            const uint32_t idesc = idesc_bf16(BM, BN);
            bool ok = true;
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % STAGES;
                if (!mbar_wait(&full[s], (kb / STAGES) & 1)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t a0 = smem_u32(sA + s * C::A_BYTES), b0 = smem_u32(sB + s * C::B_BYTES);
#pragma unroll
                for (int k = 0; k < BK / 16; ++k)
                    umma_bf16(tmem, sdesc_sw128(a0 + k * 32), sdesc_sw128(b0 + k * 32), idesc,
                              (kb > 0 || k > 0) ? 1u : 0u);
                umma_commit(&empty[s]);
            }
            if (!ok) {
                set_status(status, TNET_ERR_TIMEOUT);
                *abort_flag = 1;
            }
            umma_commit(done);
        }
    } else {  // epilogue warps 2..5
        const int q = warp & 3;
        const bool ok = mbar_wait(done, 0);
        fence_after();
        if (!ok) set_status(status, TNET_ERR_TIMEOUT);
        if (ok && !*abort_flag) {
            const int row = m0 + 32 * q + lane;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
                if (row < M) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int n = n0 + c0 + 4 * j;
                        if (n < P.N) epi(z, P.row0[z] + row, n, &v[4 * j]);
                    }
                }
            }
        }
    }
    fence_before();
    __syncthreads();
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

// 2-D bf16 tensor map: `rows` rows of `cols` elements, row pitch `ld`
// elements, box of `box_rows` x 64 elements, 128B swizzle, zero fill.
int make_map_bf16(CUtensorMap *m, const void *base, int64_t rows, int64_t cols, int64_t ld, int box_rows);

template <int BN, class Epi>
int tc_gemm(const TcShape &P, const __nv_bfloat16 *A, int64_t a_rows, int64_t lda, const __nv_bfloat16 *B,
            int64_t b_rows, int64_t ldb, const Epi &epi, int32_t *status, cudaStream_t st) {
    using C = TileCfg<BN>;
    int maxM = 0;
    for (int z = 0; z < P.nclass; ++z) maxM = P.M[z] > maxM ? P.M[z] : maxM;
    if (maxM <= 0 || P.N <= 0) return TNET_OK;
    if (P.N % 4 || (lda * 2) % 16 || (ldb * 2) % 16 || ((uintptr_t)A & 15) || ((uintptr_t)B & 15))
        return TNET_ERR_ARG;
    CUtensorMap ma, mb;
    int rc = make_map_bf16(&ma, A, a_rows, P.K, lda, BM);
    if (rc) return rc;
    rc = make_map_bf16(&mb, B, b_rows, P.K, ldb, BN);
    if (rc) return rc;
    static bool attr_set = false;
    if (!attr_set) {
        TNET_CUDA_TRY(cudaFuncSetAttribute(k_tc_gemm<BN, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)C::SMEM));
        attr_set = true;
    }
    dim3 g((maxM + BM - 1) / BM, (P.N + BN - 1) / BN, P.nclass);
    k_tc_gemm<BN, Epi><<<g, THREADS, C::SMEM, st>>>(ma, mb, P, epi, status);
    count_launch();
    TNET_LAUNCH_CHECK();
    return TNET_OK;
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
