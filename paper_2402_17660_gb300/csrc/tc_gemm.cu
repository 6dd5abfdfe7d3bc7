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

int make_map_bf16(CUtensorMap *m, const void *base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
    EncodeFn enc = tensor_map_encoder();
    if (!enc) return TNET_ERR_CUDA;
    if (rows < 1 || cols < 1 || box_rows < 1 || box_rows > 256) return TNET_ERR_ARG;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        fprintf(stderr, "libtnet: cuTensorMapEncodeTiled failed (%d)\n", (int)r);
        return TNET_ERR_CUDA;
    }
    return TNET_OK;
}

}  // namespace tc
}  // namespace tnet

using namespace tnet;

extern "C" int tnet_debug_tc_gemm(int M, int N, int K, const void *A, const void *B, float *Cout, int32_t *status,
                                  tnet_stream_t stream) {
    if (M < 1 || N < 4 || N > 512 || K < 8 || K % 8 || N % 4 || !A || !B || !Cout) return TNET_ERR_ARG;
    tc::TcShape P = tc::tshape(M, N, K);
    EpiStore epi{Cout, N, 0};
    const __nv_bfloat16 *a = (const __nv_bfloat16 *)A, *b = (const __nv_bfloat16 *)B;
    cudaStream_t st = (cudaStream_t)stream;
    if (N <= 32) return tc::tc_gemm<32>(P, a, M, K, b, N, K, epi, status, st);
    if (N <= 64) return tc::tc_gemm<64>(P, a, M, K, b, N, K, epi, status, st);
    if (N <= 128) return tc::tc_gemm<128>(P, a, M, K, b, N, K, epi, status, st);
    if (N % 192 == 0) return tc::tc_gemm<192>(P, a, M, K, b, N, K, epi, status, st);
    return tc::tc_gemm<256>(P, a, M, K, b, N, K, epi, status, st);
}
