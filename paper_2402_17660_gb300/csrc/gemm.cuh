// FP32 SIMT GEMM with fused epilogues, used for the per-atom and per-edge
// dense layers of the FP32 path.
//
//   C[m][n] = epi( sum_k A(m,k) B(k,n) )
//   A(m,k) = TA ? A[k*lda + m] : A[m*lda + k]
//   B(k,n) = TB ? B[n*ldb + k] : B[k*ldb + n]      (TB: weights stored (out, in))
//
// Up to 3 "classes" (blockIdx.z) share one launch: class z uses rows
// [row0[z], row0[z] + rows[z]) of A and C and the weight B + z*strideB.
// This is how one launch mixes the I, A and S coordinate planes with their
// own matrices.  The row count of a class may be read from device memory
// (rows_dev, times rows_mul), so launches sized for a capacity stay valid
// inside a CUDA graph when the true count is only known on the device.
// Tiles are visited by a persistent grid-stride loop.
#pragma once
#include <cuda_bf16.h>

#include "internal.cuh"

namespace tnet {

constexpr int GBM = 128, GBN = 64, GBK = 8, GTHREADS = 256;

struct GemmShape {
    int M[3];                // rows per class (capacity when rows_dev is set)
    int64_t row0[3];         // first row of each class in A and C
    const int32_t *rows_dev; // optional device row count (applies to class 0 only)
    int rows_mul;
    int N, K;
    const float *A;
    int64_t lda;
    const float *B;
    int64_t ldb, strideB;
    int nclass;
};

// --------------------------------------------------------------- epilogues
// Each epilogue receives 4 consecutive columns (n..n+3, all < N) of row m by
// value (a pointer would force the accumulator fragment into local memory).
// Optional bf16 operand copies feed the BF16 tensor-core GEMMs.
__device__ __forceinline__ void store_copy4(const OpCopy &c, int64_t idx, const float o[4]) {
    if (c.mode == 1) {
        __nv_bfloat162 a = __floats2bfloat162_rn(o[0], o[1]), b = __floats2bfloat162_rn(o[2], o[3]);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t *>(&a);
        u.y = *reinterpret_cast<uint32_t *>(&b);
        *reinterpret_cast<uint2 *>(static_cast<__nv_bfloat16 *>(c.p) + idx) = u;
    }
}

// Each functor splits into pre() (the loads: issued for several rows before
// the accumulator values arrive, so their latency overlaps) and post() (the
// arithmetic and stores); operator() runs both.  pre() may be given a row or
// column clamped into range, and its result is then unused.
struct EpiStore {  // C = v (+ C when accumulate)
    float *C;
    int64_t ldc;
    int accumulate;
    struct Pre {
        float4 c;
    };
    __device__ Pre pre(int, int64_t m, int n) const {
        return Pre{accumulate ? *reinterpret_cast<const float4 *>(C + m * ldc + n) : make_float4(0.f, 0.f, 0.f, 0.f)};
    }
    __device__ void post(int, int64_t m, int n, float4 o, const Pre &p) const {
        if (accumulate) {
            o.x += p.c.x; o.y += p.c.y; o.z += p.c.z; o.w += p.c.w;
        }
        *reinterpret_cast<float4 *>(C + m * ldc + n) = o;
    }
    __device__ void operator()(int z, int64_t m, int n, float4 o) const { post(z, m, n, o, pre(z, m, n)); }
};

struct EpiBiasAct {  // a = v + bias; pre = a; out = act(a) * rowscale[m] (+ operand copy)
    const float *bias;
    float *pre_out;
    int64_t ldp;
    float *out;
    int64_t ldo;
    int silu;
    const float *rowscale;
    OpCopy out_cp;
    int64_t ldoc;
    struct Pre {
        float4 b;
        float rs;
    };
    __device__ Pre pre(int, int64_t m, int n) const {
        return Pre{bias ? *reinterpret_cast<const float4 *>(bias + n) : make_float4(0.f, 0.f, 0.f, 0.f),
                   rowscale ? rowscale[m] : 1.0f};
    }
    __device__ void post(int, int64_t m, int n, float4 vv, const Pre &p) const {
        const float v[4] = {vv.x, vv.y, vv.z, vv.w};
        const float bv[4] = {p.b.x, p.b.y, p.b.z, p.b.w};
        float a[4], o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            a[q] = v[q] + bv[q];
            o[q] = (silu ? silu_f(a[q]) : a[q]) * p.rs;
        }
        if (pre_out) *reinterpret_cast<float4 *>(pre_out + m * ldp + n) = make_float4(a[0], a[1], a[2], a[3]);
        if (out) *reinterpret_cast<float4 *>(out + m * ldo + n) = make_float4(o[0], o[1], o[2], o[3]);
        if (out_cp.mode) store_copy4(out_cp, m * ldoc + n, o);
    }
    __device__ void operator()(int z, int64_t m, int n, float4 o) const { post(z, m, n, o, pre(z, m, n)); }
};

struct EpiGradAct {  // out = v * silu'(pre)  (+ out when accumulate) (+ operand copy)
    const float *pre_in;
    int64_t ldp;
    float *out;
    int64_t ldo;
    int accumulate;
    OpCopy out_cp;
    int64_t ldoc;
    struct Pre {
        float4 a, c;
    };
    __device__ Pre pre(int, int64_t m, int n) const {
        return Pre{*reinterpret_cast<const float4 *>(pre_in + m * ldp + n),
                   accumulate ? *reinterpret_cast<const float4 *>(out + m * ldo + n) : make_float4(0.f, 0.f, 0.f, 0.f)};
    }
    __device__ void post(int, int64_t m, int n, float4 vv, const Pre &p) const {
        float o[4] = {vv.x * silu_grad_f(p.a.x), vv.y * silu_grad_f(p.a.y), vv.z * silu_grad_f(p.a.z),
                      vv.w * silu_grad_f(p.a.w)};
        if (accumulate) {
            o[0] += p.c.x; o[1] += p.c.y; o[2] += p.c.z; o[3] += p.c.w;
        }
        *reinterpret_cast<float4 *>(out + m * ldo + n) = make_float4(o[0], o[1], o[2], o[3]);
        if (out_cp.mode) store_copy4(out_cp, m * ldoc + n, o);
    }
    __device__ void operator()(int z, int64_t m, int n, float4 o) const { post(z, m, n, o, pre(z, m, n)); }
};

// --------------------------------------------------------------- kernel ---
template <bool TA, bool TB, class Epi>
__global__ void __launch_bounds__(GTHREADS) k_sgemm(GemmShape P, Epi epi) {
    pdl_entry();
    __shared__ __align__(16) float As[2][GBK][GBM];
    __shared__ __align__(16) float Bs[2][GBK][GBN];
    const int z = blockIdx.z;
    // selects, not P.M[z]: a dynamically indexed parameter array is copied to local memory
    int M = z == 0 ? P.M[0] : (z == 1 ? P.M[1] : P.M[2]);
    if (z == 0 && P.rows_dev) {
        const int md = *P.rows_dev * P.rows_mul;
        M = md < M ? md : M;
    }
    const int64_t r0 = z == 0 ? P.row0[0] : (z == 1 ? P.row0[1] : P.row0[2]);
    const float *A = P.A + (TA ? r0 : r0 * P.lda);
    const float *B = P.B + (int64_t)z * P.strideB;
    const int N = P.N, K = P.K;
    const int tilesN = (N + GBN - 1) / GBN;
    const int tilesM = (M + GBM - 1) / GBM;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;  // 16 x 16 threads, 8x4 outputs each

    for (int tile = blockIdx.x; tile < tilesM * tilesN; tile += gridDim.x) {
        const int tm = tile / tilesN, tn = tile % tilesN;
        const int m0 = tm * GBM, n0 = tn * GBN;
        float acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

        // global -> register staging
        float4 ra, rb;
        auto load_a = [&](int k0) {
            if (!TA) {  // A[m][k]: thread loads row m0 + tid/2, k0 + (tid&1)*4
                const int m = m0 + (tid >> 1), k = k0 + (tid & 1) * 4;
                ra = (m < M) ? *reinterpret_cast<const float4 *>(A + (int64_t)m * P.lda + k)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
            } else {    // A[k][m]: thread loads k0 + tid/32, m0 + (tid&31)*4
                const int k = k0 + (tid >> 5), m = m0 + (tid & 31) * 4;
                ra = make_float4(0.f, 0.f, 0.f, 0.f);
                const float *p = A + (int64_t)k * P.lda + m;
                if (m + 3 < M) ra = *reinterpret_cast<const float4 *>(p);
                else {
                    if (m < M) ra.x = p[0];
                    if (m + 1 < M) ra.y = p[1];
                    if (m + 2 < M) ra.z = p[2];
                }
            }
        };
        auto load_b = [&](int k0) {
            if (tid >= 128) return;
            if (TB) {  // B[n][k]: thread loads n0 + tid/2, k0 + (tid&1)*4
                const int n = n0 + (tid >> 1), k = k0 + (tid & 1) * 4;
                rb = (n < N) ? *reinterpret_cast<const float4 *>(B + (int64_t)n * P.ldb + k)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
            } else {   // B[k][n]: thread loads k0 + tid/16, n0 + (tid&15)*4
                const int k = k0 + (tid >> 4), n = n0 + (tid & 15) * 4;
                rb = (n < N) ? *reinterpret_cast<const float4 *>(B + (int64_t)k * P.ldb + n)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        auto store_ab = [&](int buf) {
            if (!TA) {
                const int m = tid >> 1, k = (tid & 1) * 4;
                As[buf][k][m] = ra.x; As[buf][k + 1][m] = ra.y; As[buf][k + 2][m] = ra.z; As[buf][k + 3][m] = ra.w;
            } else {
                const int k = tid >> 5, m = (tid & 31) * 4;
                *reinterpret_cast<float4 *>(&As[buf][k][m]) = ra;
            }
            if (tid < 128) {
                if (TB) {
                    const int n = tid >> 1, k = (tid & 1) * 4;
                    Bs[buf][k][n] = rb.x; Bs[buf][k + 1][n] = rb.y; Bs[buf][k + 2][n] = rb.z; Bs[buf][k + 3][n] = rb.w;
                } else {
                    const int k = tid >> 4, n = (tid & 15) * 4;
                    *reinterpret_cast<float4 *>(&Bs[buf][k][n]) = rb;
                }
            }
        };

        load_a(0);
        load_b(0);
        store_ab(0);
        __syncthreads();
        int buf = 0;
        for (int k0 = 0; k0 < K; k0 += GBK) {
            const bool more = k0 + GBK < K;
            if (more) {
                load_a(k0 + GBK);
                load_b(k0 + GBK);
            }
#pragma unroll
            for (int kk = 0; kk < GBK; ++kk) {
                const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 8]);
                const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 8 + 4]);
                const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
                const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bv[4] = {b0.x, b0.y, b0.z, b0.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
            if (more) {
                store_ab(buf ^ 1);
                __syncthreads();
                buf ^= 1;
            }
        }
        // epilogue
        const int n = n0 + tx * 4;
        if (n < N) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int m = m0 + ty * 8 + i;
                if (m < M) epi(z, r0 + m, n, make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]));
            }
        }
        __syncthreads();
    }
}

// Host launcher.  grid: persistent, sized from the capacity.
// max_ctas: size of the persistent grid (a tuning knob: SMs x CTAs per SM)
template <bool TA, bool TB, class Epi>
inline int sgemm(const GemmShape &P, const Epi &epi, int max_ctas, cudaStream_t st) {
    int maxM = 0;
    for (int z = 0; z < P.nclass; ++z) maxM = P.M[z] > maxM ? P.M[z] : maxM;
    if (maxM <= 0 || P.N <= 0) return TNET_OK;
    if (P.K % GBK || P.N % 4) return TNET_ERR_ARG;
    const int64_t tiles = (int64_t)((maxM + GBM - 1) / GBM) * ((P.N + GBN - 1) / GBN);
    int64_t grid = max_ctas > 0 ? max_ctas : 1;
    if (tiles < grid) grid = tiles;
    dim3 g((unsigned)grid, 1, P.nclass);
    launch(k_sgemm<TA, TB, Epi>, g, GTHREADS, 0, st, P, epi);
    count_launch();
    TNET_LAUNCH_CHECK();
    return TNET_OK;
}

inline GemmShape gshape(int M, int N, int K, const float *A, int64_t lda, const float *B, int64_t ldb) {
    GemmShape P{};
    P.M[0] = M;
    P.row0[0] = 0;
    P.rows_dev = nullptr;
    P.rows_mul = 1;
    P.N = N;
    P.K = K;
    P.A = A;
    P.lda = lda;
    P.B = B;
    P.ldb = ldb;
    P.strideB = 0;
    P.nclass = 1;
    return P;
}

// The three coordinate classes of a node tensor buffer with N atoms:
// I rows [0, N), A rows [N, 4N), S rows [4N, 9N); weights W[3][F][F].
inline GemmShape gshape_classes(int N, int F, const float *A, const float *W) {
    GemmShape P{};
    P.M[0] = N; P.M[1] = 3 * N; P.M[2] = 5 * N;
    P.row0[0] = 0; P.row0[1] = N; P.row0[2] = 4LL * N;
    P.rows_dev = nullptr;
    P.rows_mul = 1;
    P.N = F;
    P.K = F;
    P.A = A;
    P.lda = F;
    P.B = W;
    P.ldb = F;
    P.strideB = (int64_t)F * F;
    P.nclass = 3;
    return P;
}

}  // namespace tnet
