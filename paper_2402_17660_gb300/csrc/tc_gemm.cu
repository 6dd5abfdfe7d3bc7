// Host side of the tcgen05 GEMM: tensor-map encoding and a test entry point.
#include "gemm.cuh"
#include "tc_gemm.cuh"

namespace tnet {
namespace tc {

EncodeFn tensor_map_encoder() {
    static EncodeFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeFn)p;
    }
    return fn;
}

static int make_map(CUtensorMap *m, CUtensorMapDataType dt, int esz, const void *base, int64_t rows, int64_t cols,
                    int64_t ld, int box_rows, int row_bytes) {
    EncodeFn enc = tensor_map_encoder();
    if (!enc) return TNET_ERR_CUDA;
    if (rows < 1 || cols < 1 || box_rows < 1 || box_rows > 256 || (row_bytes != 128 && row_bytes != 64))
        return TNET_ERR_ARG;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * esz)};
    cuuint32_t box[2] = {(cuuint32_t)(row_bytes / esz), (cuuint32_t)box_rows};  // rows of row_bytes
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        fprintf(stderr, "libtnet: cuTensorMapEncodeTiled failed (%d)\n", (int)r);
        return TNET_ERR_CUDA;
    }
    return TNET_OK;
}

int make_map_bf16(CUtensorMap *m, const void *base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
    return make_map(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, rows, cols, ld, box_rows, 128);
}
int make_map_f32(CUtensorMap *m, const void *base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                 int row_bytes) {
    return make_map(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, rows, cols, ld, box_rows, row_bytes);
}

}  // namespace tc
}  // namespace tnet

using namespace tnet;

// TF32 split of the weights (for the test entry point)
__global__ void k_tf32_split(const float *__restrict__ x, float *__restrict__ hi, float *__restrict__ lo, int64_t n) {
    pdl_entry();
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) tf32_split(x[t], hi[t], lo[t]);
}

// SM count of the current device (the debug entry points have no context)
static int current_sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

static int debug_f32(int M, int N, int K, const float *A, const float *B, float *Bsplit, float *Cout,
                     int32_t *status, tnet_stream_t stream, uint32_t spin_limit, int skip_mma, int cl = 1) {
    if (M < 1 || N < 4 || N > 512 || K < 4 || K % 4 || N % 4 || !A || !B || !Bsplit || !Cout) return TNET_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nk = (int64_t)N * K;
    launch(k_tf32_split, (int)((nk + 255) / 256), 256, 0, st, B, Bsplit, Bsplit + nk, nk);
    TNET_LAUNCH_CHECK();
    tc::TcShape P = tc::tshape(M, N, K);
    P.spin_limit = spin_limit;
    P.skip_mma = skip_mma;
    P.cl = cl;
    EpiStore epi{Cout, N, 0};
    const tc::TcOperands o{A, Bsplit, Bsplit + nk, M, K, N, K};
    const int sms = current_sms();
    // the library's routing: num_rbf-deep GEMMs (K <= 32) keep the 16-warp
    // epilogue and four stages
    if (N <= 32) return tc::tc_gemm_ops<32, true>(P, o, epi, status, st, sms);
    if (N <= 64) return tc::tc_gemm_ops<64, true>(P, o, epi, status, st, sms);
    if (K <= 32) {
        if (N % 192 == 0) return tc::tc_gemm_ops<192, true, true>(P, o, epi, status, st, sms);
        return tc::tc_gemm_ops<128, true, true>(P, o, epi, status, st, sms);
    }
    if (N % 256 == 0) return tc::tc_gemm_ops<256, true>(P, o, epi, status, st, sms);
    if (N % 192 == 0) return tc::tc_gemm_ops<192, true>(P, o, epi, status, st, sms);
    return tc::tc_gemm_ops<128, true>(P, o, epi, status, st, sms);
}

extern "C" int tnet_debug_tc_gemm_f32(int M, int N, int K, const float *A, const float *B, float *Bsplit, float *Cout,
                                      int32_t *status, tnet_stream_t stream) {
    return debug_f32(M, N, K, A, B, Bsplit, Cout, status, stream, 0, 0);
}

extern "C" int tnet_debug_tc_gemm_timeout(int M, int N, int K, const float *A, const float *B, float *Bsplit,
                                          float *Cout, uint32_t spin_limit, int32_t *status, tnet_stream_t stream) {
    if (spin_limit < 1) return TNET_ERR_ARG;
    return debug_f32(M, N, K, A, B, Bsplit, Cout, status, stream, spin_limit, 1);
}

static int debug_bf16(int M, int N, int K, const void *A, const void *B, float *Cout, int32_t *status,
                      tnet_stream_t stream, int cl) {
    if (M < 1 || N < 4 || N > 512 || K < 8 || K % 8 || N % 4 || !A || !B || !Cout) return TNET_ERR_ARG;
    tc::TcShape P = tc::tshape(M, N, K);
    P.cl = cl;
    EpiStore epi{Cout, N, 0};
    const __nv_bfloat16 *a = (const __nv_bfloat16 *)A, *b = (const __nv_bfloat16 *)B;
    cudaStream_t st = (cudaStream_t)stream;
    const int sms = current_sms();
    if (N <= 32) return tc::tc_gemm<32>(P, a, M, K, b, N, K, epi, status, st, sms);
    if (N <= 64) return tc::tc_gemm<64>(P, a, M, K, b, N, K, epi, status, st, sms);
    if (N <= 128) return tc::tc_gemm<128>(P, a, M, K, b, N, K, epi, status, st, sms);
    if (N % 192 == 0) return tc::tc_gemm<192>(P, a, M, K, b, N, K, epi, status, st, sms);
    return tc::tc_gemm<256>(P, a, M, K, b, N, K, epi, status, st, sms);
}

extern "C" int tnet_debug_tc_gemm(int M, int N, int K, const void *A, const void *B, float *Cout, int32_t *status,
                                  tnet_stream_t stream) {
    return debug_bf16(M, N, K, A, B, Cout, status, stream, 1);
}

extern "C" int tnet_debug_tc_gemm_cluster(int M, int N, int K, int x3, int cluster, const void *A, const void *B,
                                          float *B_split, float *Cout, int32_t *status, tnet_stream_t stream) {
    if (cluster != 1 && cluster != 2 && cluster != 4) return TNET_ERR_ARG;
    if (x3)
        return debug_f32(M, N, K, (const float *)A, (const float *)B, B_split, Cout, status, stream, 0, 0, cluster);
    return debug_bf16(M, N, K, A, B, Cout, status, stream, cluster);
}
