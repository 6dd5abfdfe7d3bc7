// Weight-gradient reductions: sums over rows (atoms, coordinate rows or
// undirected pairs) of outer products, column sums and LayerNorm parameter
// gradients.  Every reduction is split over row ranges into partial sums
// that a second kernel adds in a fixed order, so weight gradients are
// deterministic (no floating-point atomics).
#include "internal.cuh"

namespace tnet {

constexpr int WBM = 64, WBN = 64, WBK = 16, WTHREADS = 256;

// partial[(z*splits + s)][m][n] = sum over rows r of split s of A[r][m] B[r][n]
__global__ void __launch_bounds__(WTHREADS) k_wgrad(WgradShape P, int splits, int64_t chunk,
                                                    float *__restrict__ partial) {
    pdl_entry();
    __shared__ __align__(16) float As[WBK][WBM];
    __shared__ __align__(16) float Bs[WBK][WBN];
    const int z = blockIdx.z, s = blockIdx.y;
    int64_t R = z == 0 ? P.rows[0] : (z == 1 ? P.rows[1] : P.rows[2]);
    if (z == 0 && P.rows_dev) {
        const int64_t rd = (int64_t)(*P.rows_dev) * P.rows_mul;
        R = rd < R ? rd : R;
    }
    const int tilesN = (P.N + WBN - 1) / WBN;
    const int tm = blockIdx.x / tilesN, tn = blockIdx.x % tilesN;
    const int m0 = tm * WBM, n0 = tn * WBN;
    const int64_t r_begin = s * chunk;
    int64_t r_end = r_begin + chunk;
    if (r_end > R) r_end = R;
    const int64_t rz = z == 0 ? P.row0[0] : (z == 1 ? P.row0[1] : P.row0[2]);
    const float *A = P.A + rz * P.lda;
    const float *B = P.B + rz * P.ldb;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    float acc[4][4] = {};
    for (int64_t r0 = r_begin; r0 < r_end; r0 += WBK) {
        {   // 16 rows x 64 columns of A and B, one float4 each per thread
            const int rr = tid >> 4, cc = (tid & 15) * 4;
            const int64_t r = r0 + rr;
            float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = va;
            if (r < r_end) {
                if (m0 + cc < P.M) va = *reinterpret_cast<const float4 *>(A + r * P.lda + m0 + cc);
                if (n0 + cc < P.N) vb = *reinterpret_cast<const float4 *>(B + r * P.ldb + n0 + cc);
            }
            *reinterpret_cast<float4 *>(&As[rr][cc]) = va;
            *reinterpret_cast<float4 *>(&Bs[rr][cc]) = vb;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < WBK; ++k) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    float *out = partial + ((int64_t)z * splits + s) * P.M * P.N;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= P.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n < P.N) out[(int64_t)m * P.N + n] = acc[i][j];
        }
    }
}

// partial[(z*splits + s)][m] = sum over rows of split s of A[r][m] (* w[r])
__global__ void k_colsum(WgradShape P, int splits, int64_t chunk, const float *__restrict__ roww,
                         float *__restrict__ partial) {
    pdl_entry();
    const int z = blockIdx.z, s = blockIdx.y;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= P.M) return;
    int64_t R = z == 0 ? P.rows[0] : (z == 1 ? P.rows[1] : P.rows[2]);
    if (z == 0 && P.rows_dev) {
        const int64_t rd = (int64_t)(*P.rows_dev) * P.rows_mul;
        R = rd < R ? rd : R;
    }
    const int64_t r_begin = s * chunk;
    int64_t r_end = r_begin + chunk;
    if (r_end > R) r_end = R;
    const float *A = P.A + (z == 0 ? P.row0[0] : (z == 1 ? P.row0[1] : P.row0[2])) * P.lda;
    float acc = 0.f;
    for (int64_t r = r_begin; r < r_end; ++r) acc += A[r * P.lda + m] * (roww ? roww[r] : 1.0f);
    partial[((int64_t)z * splits + s) * P.M + m] = acc;
}

// LayerNorm parameter gradients: dgamma[c] = sum_r gy[r][c] xhat[r][c],
// dbeta[c] = sum_r gy[r][c], xhat = (x - mean_r) * rstd_r
__global__ void k_ln_grad(const float *__restrict__ gy, const float *__restrict__ x,
                          const float2 *__restrict__ stats, int R, int C, int splits, int64_t chunk,
                          float *__restrict__ partial) {
    pdl_entry();
    const int s = blockIdx.y;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int64_t r_begin = s * chunk;
    int64_t r_end = r_begin + chunk;
    if (r_end > R) r_end = R;
    float ag = 0.f, ab = 0.f;
    for (int64_t r = r_begin; r < r_end; ++r) {
        const float g = gy[r * C + c];
        const float2 st = stats[r];
        ag = fmaf(g, (x[r * C + c] - st.x) * st.y, ag);
        ab += g;
    }
    partial[(int64_t)s * 2 * C + c] = ag;
    partial[(int64_t)s * 2 * C + C + c] = ab;
}

// out[z][i] = sum_s partial[z][s][i]  (fixed order; + out when accumulate).
// With perm_f > 0 the rows m of each [3 perm_f][ncols] class come in
// plane-major order (m = p perm_f + c) and are written to row c*3 + p.
__global__ void k_split_reduce(const float *__restrict__ partial, int splits, int64_t per_class, int nclass,
                               float *__restrict__ out, int accumulate, int ncols, int perm_f) {
    pdl_entry();
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= per_class * nclass) return;
    const int64_t z = t / per_class, i = t % per_class;
    int64_t o = t;
    if (perm_f > 0) {
        const int64_t m = i / ncols, n = i % ncols;
        o = z * per_class + ((m % perm_f) * 3 + m / perm_f) * ncols + n;
    }
    float acc = accumulate ? out[o] : 0.f;
    const float *p = partial + z * splits * per_class + i;
    for (int s = 0; s < splits; ++s) acc += p[(int64_t)s * per_class];
    out[o] = acc;
}

static int choose_splits(int64_t rows_cap, int64_t tiles, int nclass, int64_t per_split_floats,
                         int64_t partial_cap, int sms, int64_t *chunk) {
    int64_t splits = (3LL * sms + tiles * nclass - 1) / (tiles * nclass);
    if (splits < 1) splits = 1;
    const int64_t max_by_rows = (rows_cap + 63) / 64;
    if (splits > max_by_rows) splits = max_by_rows > 0 ? max_by_rows : 1;
    const int64_t max_by_mem = partial_cap / (per_split_floats * nclass);
    if (splits > max_by_mem) splits = max_by_mem;
    if (splits < 1) splits = 1;
    *chunk = (rows_cap + splits - 1) / splits;
    *chunk = (*chunk + WBK - 1) / WBK * WBK;
    if (*chunk < WBK) *chunk = WBK;
    return (int)splits;
}

int wgrad_outer(const WgradShape &P, float *partial, int64_t partial_cap, float *out, int accumulate, int sms,
                cudaStream_t st, int perm_f) {
    int64_t rows_cap = 0;
    for (int z = 0; z < P.nclass; ++z) rows_cap = P.rows[z] > rows_cap ? P.rows[z] : rows_cap;
    if (rows_cap <= 0 || P.M <= 0 || P.N <= 0) return TNET_OK;
    if (P.M % 4 || P.N % 4 || P.lda % 4 || P.ldb % 4) return TNET_ERR_ARG;
    const int64_t tiles = (int64_t)((P.M + WBM - 1) / WBM) * ((P.N + WBN - 1) / WBN);
    int64_t chunk;
    const int splits = choose_splits(rows_cap, tiles, P.nclass, (int64_t)P.M * P.N, partial_cap, sms, &chunk);
    if ((int64_t)splits * P.nclass * P.M * P.N > partial_cap) return TNET_ERR_WORKSPACE;
    dim3 g((unsigned)tiles, splits, P.nclass);
    launch(k_wgrad, g, WTHREADS, 0, st, P, splits, chunk, partial);
    count_launch();
    const int64_t tot = (int64_t)P.nclass * P.M * P.N;
    launch(k_split_reduce, (unsigned)((tot + 255) / 256), 256, 0, st, partial, splits, (int64_t)P.M * P.N, P.nclass,
                                                                  out, accumulate, P.N, perm_f);
    count_launch();
    TNET_LAUNCH_CHECK();
    return TNET_OK;
}

int wgrad_colsum(const WgradShape &P, const float *roww, float *partial, int64_t partial_cap, float *out,
                 int accumulate, int sms, cudaStream_t st, int perm_f) {
    int64_t rows_cap = 0;
    for (int z = 0; z < P.nclass; ++z) rows_cap = P.rows[z] > rows_cap ? P.rows[z] : rows_cap;
    if (rows_cap <= 0 || P.M <= 0) return TNET_OK;
    const int64_t tiles = (P.M + 255) / 256;
    int64_t chunk;
    const int splits = choose_splits(rows_cap, tiles * 4, P.nclass, P.M, partial_cap, sms, &chunk);
    dim3 g((unsigned)tiles, splits, P.nclass);
    launch(k_colsum, g, 256, 0, st, P, splits, chunk, roww, partial);
    count_launch();
    const int64_t tot = (int64_t)P.nclass * P.M;
    launch(k_split_reduce, (unsigned)((tot + 255) / 256), 256, 0, st, partial, splits, P.M, P.nclass, out, accumulate,
                                                                  1, perm_f);
    count_launch();
    TNET_LAUNCH_CHECK();
    return TNET_OK;
}

// out_g[0..C) = dgamma, out_g[C..2C) = dbeta (gamma and beta are adjacent in
// the weight blob)
int wgrad_layernorm(const float *gy, const float *x, const float2 *stats, int R, int C, float *partial,
                    int64_t partial_cap, float *out_g, int sms, cudaStream_t st) {
    if (R <= 0) return TNET_OK;
    const int64_t tiles = (C + 255) / 256;
    int64_t chunk;
    const int splits = choose_splits(R, tiles * 4, 1, 2LL * C, partial_cap, sms, &chunk);
    dim3 g((unsigned)tiles, splits, 1);
    launch(k_ln_grad, g, 256, 0, st, gy, x, stats, R, C, splits, chunk, partial);
    count_launch();
    launch(k_split_reduce, (unsigned)((2 * C + 255) / 256), 256, 0, st, partial, splits, 2LL * C, 1, out_g, 0, 1, 0);
    count_launch();
    TNET_LAUNCH_CHECK();
    return TNET_OK;
}

}  // namespace tnet
