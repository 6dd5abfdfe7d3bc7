// Internal definitions shared by the libtnet CUDA sources.
#pragma once
#include <utility>

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/tnet.h"

#define TNET_CUDA_TRY(expr)                                                         \
    do {                                                                            \
        cudaError_t e_ = (expr);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            fprintf(stderr, "libtnet: %s failed: %s (%s:%d)\n", #expr,              \
                    cudaGetErrorString(e_), __FILE__, __LINE__);                    \
            return TNET_ERR_CUDA;                                                   \
        }                                                                           \
    } while (0)

#define TNET_LAUNCH_CHECK() TNET_CUDA_TRY(cudaGetLastError())

namespace tnet {

// Programmatic dependent launch.  Kernels of the library are launched (unless
// the context's pdl knob is 0) with the programmatic-serialization attribute,
// so the next kernel of a
// stream (or graph) may be scheduled while the previous one drains; its first
// statement, pdl_entry(), waits until the previous grid has completed and its
// writes are visible (griddepcontrol.wait), then lets the following kernel be
// scheduled once all of this grid's CTAs are running.  Without a programmatic
// predecessor both instructions are no-ops.
__device__ __forceinline__ void pdl_entry() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// Whether launches of this host thread carry the attribute: set for the
// duration of each API call from the context's tuning knob (PdlScope).
extern thread_local int tl_pdl;
struct PdlScope {
    int prev;
    explicit PdlScope(int on) : prev(tl_pdl) { tl_pdl = on; }
    ~PdlScope() { tl_pdl = prev; }
};
template <typename... KArgs, typename... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = tl_pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);  // errors surface in cudaGetLastError
}

// The same with a 1-D thread-block cluster of `cluster` CTAs (1: none).
template <typename... KArgs, typename... Args>
inline void launch_cluster(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, int cluster,
                           Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    int n = 0;
    if (cluster > 1) {
        attr[n].id = cudaLaunchAttributeClusterDimension;
        attr[n].val.clusterDim.x = (unsigned)cluster;
        attr[n].val.clusterDim.y = 1;
        attr[n].val.clusterDim.z = 1;
        ++n;
    }
    if (tl_pdl) {
        attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[n].val.programmaticStreamSerializationAllowed = 1;
        ++n;
    }
    cfg.attrs = attr;
    cfg.numAttrs = n;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);  // errors surface in cudaGetLastError
}

constexpr int kMaxCellsPerAtom = 2;   // cell budget: 2 cells per atom + 8 per system + 64
constexpr int kMaxRowSorted = 1024;   // longest CSR row sorted in shared memory
constexpr int kSlabWidth = 128;       // columns per atom in the single-pass search's row slab

// First device-detected error wins.
__device__ __forceinline__ void set_status(int32_t *st, int code) {
    if (st) atomicCAS(st, 0, code);
}

// Per-system cell grid (one cell list per system; cells never mix systems).
struct SysInfo {
    float origin[3];    // no PBC: lower corner of the grid
    float inv_cell[3];  // no PBC: 1 / cell width along x, y, z
    float L[3];         // PBC: box diagonal ax, by, cz; 0 when not periodic
    float tilt[3];      // PBC: bx, cx, cy of the lower-triangular box (0: rectangular)
    int nc[3];          // cells along x, y, z (PBC: along a, b, c) (>= 1)
    int cell_off;       // first global cell index of this system
    int pbc;            // 1 if periodic
    int pad;
};

// ---------------------------------------------------------------------------
// Compact rank-2 tensor coordinates.  A 3x3 feature X = i*Id + [a]_x + S is
// stored as 9 coordinates v = (i, ax, ay, az, sxx, syy, sxy, sxz, syz) with
// S symmetric-traceless (szz = -sxx - syy) and [a]_x the skew matrix with
// [a]_x w = a x w.  The I/A/S parts are coordinate groups {0}, {1,2,3},
// {4..8}; channel mixing acts on every coordinate alike.
//
// Memory layout of a node tensor buffer for N atoms and F channels: three
// row planes of F floats, I rows [0,N) (row n), A rows [N,4N) (row N+3n+k),
// S rows [4N,9N) (row 4N+5n+k).  A class-p mixing is one GEMM over a
// contiguous block of rows.
// ---------------------------------------------------------------------------
// Runs CALL(F) with F as a compile-time constant (the channel counts the
// library accepts: multiples of 64 up to 512); returns TNET_ERR_ARG otherwise.
#define TNET_F_SWITCH(Fv, CALL)                 \
    switch (Fv) {                              \
        case 64: CALL(64); break;              \
        case 128: CALL(128); break;            \
        case 192: CALL(192); break;            \
        case 256: CALL(256); break;            \
        case 320: CALL(320); break;            \
        case 384: CALL(384); break;            \
        case 448: CALL(448); break;            \
        case 512: CALL(512); break;            \
        default: return TNET_ERR_ARG;          \
    }

__device__ __forceinline__ int64_t crow(int n, int k, int N) {
    return k == 0 ? (int64_t)n : (k < 4 ? (int64_t)N + 3LL * n + (k - 1) : 4LL * N + 5LL * n + (k - 4));
}

__device__ __forceinline__ void load_coords(const float *__restrict__ T, int n, int c, int N, int F,
                                            float v[9]) {
    const float *pI = T + (int64_t)n * F + c;
    const float *pA = T + ((int64_t)N + 3LL * n) * F + c;
    const float *pS = T + (4LL * N + 5LL * n) * F + c;
    v[0] = pI[0];
#pragma unroll
    for (int k = 0; k < 3; ++k) v[1 + k] = pA[(int64_t)k * F];
#pragma unroll
    for (int k = 0; k < 5; ++k) v[4 + k] = pS[(int64_t)k * F];
}

__device__ __forceinline__ void store_coords(float *__restrict__ T, int n, int c, int N, int F,
                                             const float v[9]) {
    float *pI = T + (int64_t)n * F + c;
    float *pA = T + ((int64_t)N + 3LL * n) * F + c;
    float *pS = T + (4LL * N + 5LL * n) * F + c;
    pI[0] = v[0];
#pragma unroll
    for (int k = 0; k < 3; ++k) pA[(int64_t)k * F] = v[1 + k];
#pragma unroll
    for (int k = 0; k < 5; ++k) pS[(int64_t)k * F] = v[4 + k];
}

// Operand copy written next to an FP32 result for the BF16 tensor-core GEMMs
// (mode 1: a bf16 copy; mode 0: none).  The 3xTF32 GEMMs read the fp32
// result itself and form its TF32 residual in shared memory.
struct OpCopy {
    void *p;
    int mode;
};
// Split of an fp32 value for 3xTF32: hi = x rounded to the nearest TF32
// value (PTX cvt.rna.tf32.f32: 10 explicit mantissa bits), lo = x - hi
// (exact in fp32, |lo| <= 2^-11 |x|) rounded to TF32 in turn.  Both halves are
// TF32-representable, so the tensor core reads them exactly, and
// hi + lo = x within 2^-22 |x|.
__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
__device__ __forceinline__ void tf32_split(float x, float &hi, float &lo) {
    hi = tf32_round(x);
    lo = tf32_round(__fsub_rn(x, hi));
}
__device__ __forceinline__ void opcopy_store(const OpCopy &c, int64_t idx, float v) {
    if (c.mode == 1) static_cast<__nv_bfloat16 *>(c.p)[idx] = __float2bfloat16_rn(v);
}
__device__ __forceinline__ void store_coords_cp(const OpCopy &T, int n, int c, int N, int F, const float v[9]) {
    if (!T.mode) return;
    opcopy_store(T, (int64_t)n * F + c, v[0]);
#pragma unroll
    for (int k = 0; k < 3; ++k) opcopy_store(T, ((int64_t)N + 3LL * n + k) * F + c, v[1 + k]);
#pragma unroll
    for (int k = 0; k < 5; ++k) opcopy_store(T, (4LL * N + 5LL * n + k) * F + c, v[4 + k]);
}

// coordinates -> row-major 3x3
__device__ __forceinline__ void expand(const float v[9], float m[9]) {
    const float i = v[0], ax = v[1], ay = v[2], az = v[3];
    const float sxx = v[4], syy = v[5], sxy = v[6], sxz = v[7], syz = v[8];
    m[0] = i + sxx; m[1] = sxy - az; m[2] = sxz + ay;
    m[3] = sxy + az; m[4] = i + syy; m[5] = syz - ax;
    m[6] = sxz - ay; m[7] = syz + ax; m[8] = i - sxx - syy;
}

// row-major 3x3 -> coordinates of its I, A, S parts
__device__ __forceinline__ void decomp(const float m[9], float v[9]) {
    const float i = (m[0] + m[4] + m[8]) * (1.0f / 3.0f);
    v[0] = i;
    v[1] = 0.5f * (m[7] - m[5]);
    v[2] = 0.5f * (m[2] - m[6]);
    v[3] = 0.5f * (m[3] - m[1]);
    v[4] = m[0] - i;
    v[5] = m[4] - i;
    v[6] = 0.5f * (m[1] + m[3]);
    v[7] = 0.5f * (m[2] + m[6]);
    v[8] = 0.5f * (m[5] + m[7]);
}

// gradient w.r.t. coordinates of f(expand(v)) given G = df/dm (transpose of expand)
__device__ __forceinline__ void expand_T(const float G[9], float g[9]) {
    g[0] = G[0] + G[4] + G[8];
    g[1] = G[7] - G[5];
    g[2] = G[2] - G[6];
    g[3] = G[3] - G[1];
    g[4] = G[0] - G[8];
    g[5] = G[4] - G[8];
    g[6] = G[1] + G[3];
    g[7] = G[2] + G[6];
    g[8] = G[5] + G[7];
}

// gradient w.r.t. the matrix of f(decomp(m)) given g = df/dv (transpose of decomp)
__device__ __forceinline__ void decomp_T(const float g[9], float G[9]) {
    const float dg = (g[0] - g[4] - g[5]) * (1.0f / 3.0f);
    G[0] = dg + g[4];
    G[4] = dg + g[5];
    G[8] = dg;
    G[1] = 0.5f * (g[6] - g[3]);
    G[3] = 0.5f * (g[6] + g[3]);
    G[2] = 0.5f * (g[7] + g[2]);
    G[6] = 0.5f * (g[7] - g[2]);
    G[5] = 0.5f * (g[8] - g[1]);
    G[7] = 0.5f * (g[8] + g[1]);
}

// squared Frobenius norm of expand(v)
__device__ __forceinline__ float cnorm(const float v[9]) {
    const float sxx = v[4], syy = v[5], szz = -(v[4] + v[5]);
    return 3.0f * v[0] * v[0] + 2.0f * (v[1] * v[1] + v[2] * v[2] + v[3] * v[3]) + sxx * sxx +
           syy * syy + szz * szz + 2.0f * (v[6] * v[6] + v[7] * v[7] + v[8] * v[8]);
}

// d cnorm / d v
__device__ __forceinline__ void cnorm_grad(const float v[9], float g[9]) {
    g[0] = 6.0f * v[0];
    g[1] = 4.0f * v[1];
    g[2] = 4.0f * v[2];
    g[3] = 4.0f * v[3];
    g[4] = 4.0f * v[4] + 2.0f * v[5];
    g[5] = 4.0f * v[5] + 2.0f * v[4];
    g[6] = 4.0f * v[6];
    g[7] = 4.0f * v[7];
    g[8] = 4.0f * v[8];
}

// C = A B (row-major 3x3)
__device__ __forceinline__ void mm3(const float A[9], const float B[9], float C[9]) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            C[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
}

// C = A^T B
__device__ __forceinline__ void mm3_tn(const float A[9], const float B[9], float C[9]) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            C[3 * r + c] = A[r] * B[c] + A[3 + r] * B[3 + c] + A[6 + r] * B[6 + c];
}

// C = A B^T
__device__ __forceinline__ void mm3_nt(const float A[9], const float B[9], float C[9]) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            C[3 * r + c] = A[3 * r] * B[3 * c] + A[3 * r + 1] * B[3 * c + 1] + A[3 * r + 2] * B[3 * c + 2];
}

// Barrier of the F threads of row group g of a block holding RB groups
// (named barrier 1 + g; barrier 0 is __syncthreads); the whole block when RB = 1.
template <int F, int RB>
__device__ __forceinline__ void group_sync(int g) {
    if constexpr (RB == 1) {
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "n"(F) : "memory");
    }
}

// SiLU and its derivative (fast-math exp and divide: a few ulp, far inside
// the FP32 path's error budget)
__device__ __forceinline__ float silu_f(float x) { return __fdividef(x, 1.0f + __expf(-x)); }
__device__ __forceinline__ float silu_grad_f(float x) {
    const float s = __fdividef(1.0f, 1.0f + __expf(-x));
    return s * (1.0f + x * (1.0f - s));
}
// silu(x) and silu'(x) from one sigmoid evaluation
__device__ __forceinline__ void silu_and_grad_f(float x, float &v, float &d) {
    const float s = __fdividef(1.0f, 1.0f + __expf(-x));
    v = x * s;
    d = s * (1.0f + x * (1.0f - s));
}

// ------------------------------------------------------------- geometry ---
// Nearest periodic image of a pair vector for a rectangular box; L = 0 along
// an axis means that axis is not periodic.
// Pair geometry with every rounding fixed (the _rn intrinsics are never
// contracted into FMAs): kernels that decide the same pair independently (the
// neighbor count and fill passes, the model's upper-pair count and
// assignment) then agree even for a pair within an ulp of the cutoff, and
// r_ji is exactly -r_ij.
__device__ __forceinline__ float mic1(float x, float L) {
    return __fsub_rn(x, __fmul_rn(L, rintf(__fdiv_rn(x, L))));
}
__device__ __forceinline__ float norm2_rn(float x, float y, float z) {
    return __fadd_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)), __fmul_rn(z, z));
}
// Nearest image for a lower-triangular box with rows a = (ax,0,0),
// b = (bx,by,0), c = (cx,cy,cz): remove c round(z/cz), then b round(y/by),
// then a round(x/ax).  The result lies in the brick |x| <= ax/2, |y| <= by/2,
// |z| <= cz/2, which holds one image of every vector; since the box's
// perpendicular widths obey w_c = cz, w_b <= by, w_a <= ax, an image shorter
// than half the smallest width is that one.  Rectangular boxes have zero
// tilts, and then this is mic1 along each axis.
__device__ __forceinline__ void mic_lower(float &x, float &y, float &z, float ax, float bx, float by, float cx,
                                          float cy, float cz) {
    const float kc = rintf(__fdiv_rn(z, cz));
    x = __fsub_rn(x, __fmul_rn(kc, cx));
    y = __fsub_rn(y, __fmul_rn(kc, cy));
    z = __fsub_rn(z, __fmul_rn(kc, cz));
    const float kb = rintf(__fdiv_rn(y, by));
    x = __fsub_rn(x, __fmul_rn(kb, bx));
    y = __fsub_rn(y, __fmul_rn(kb, by));
    x = __fsub_rn(x, __fmul_rn(rintf(__fdiv_rn(x, ax)), ax));
}
// the same with the box as 9 floats, rows a, b, c
__device__ __forceinline__ void mic_box(float &x, float &y, float &z, const float *__restrict__ B) {
    mic_lower(x, y, z, B[0], B[3], B[4], B[6], B[7], B[8]);
}
__device__ __forceinline__ void mic(float &x, float &y, float &z, const SysInfo &s) {
    if (s.pbc) mic_lower(x, y, z, s.L[0], s.tilt[0], s.L[1], s.tilt[1], s.tilt[2], s.L[2]);
}

// Radial part of the model: cosine cutoff phi(d), expnorm basis e_k(d) and
// their derivatives.  Parameters precomputed on the host.
struct RadialParams {
    float rc, rl;       // cutoff_upper, cutoff_lower
    float alpha, beta;  // expnorm decay and width
    float mu0, dmu;     // centres mu_k = mu0 + k * dmu
    int K;
};

__device__ __forceinline__ float cutoff_phi(float d, const RadialParams &p) {
    return d < p.rc ? 0.5f * (cospif(d / p.rc) + 1.0f) : 0.0f;
}
__device__ __forceinline__ float cutoff_dphi(float d, const RadialParams &p) {
    return d < p.rc ? -0.5f * 3.14159265358979f / p.rc * sinpif(d / p.rc) : 0.0f;
}
// k-th basis value (including the phi factor) and its d-derivative
__device__ __forceinline__ void expnorm_k(float d, int k, const RadialParams &p, float phi, float dphi,
                                          float &e, float &de) {
    const float ex = expf(p.alpha * (p.rl - d));
    const float t = ex - (p.mu0 + k * p.dmu);
    const float rho = expf(-p.beta * t * t);
    e = phi * rho;
    de = dphi * rho + phi * rho * (2.0f * p.beta * t * p.alpha * ex);
}

// ------------------------------------------------------------ workspace ---
struct Layout {
    // neighbor search
    size_t sys_start, sys_end, sysinfo, sys_ncell, cell_count, cell_start, cell_fill, cell_of,
        sorted, spos, rowcnt, scan_tmp;
    // single-pass search: each row's sorted columns, kSlabWidth per atom, and
    // the flag of a row that did not fit (slab_width 0: two passes)
    size_t slab, slab_over;
    int slab_width;
    // energy / forces: graph bookkeeping
    size_t rev, pair_of, uedge, ucnt, nu, rp_safe;
    // node buffers
    size_t Ta, Tb, Xraw, Uemb, n0, as1, hs1, as2, s, ln0;
    size_t Xin, qn, Xn, Y, M, Tn, dX;  // per layer (stride given below)
    size_t Xfin, h, hn, lno, ao, o, at, t, Ei;
    // edge MLP (undirected active edges)
    size_t eu, phiu, geo, a1, h1, a2, h2, a3;
    // backward
    size_t gXa, gXb, gdX, gTn, gM, gY, gat, gao, ghn, gh, gU, gas2, gas1, gn0, gq0, gg, ga2, ga1, ge,
        gphiu, gvec;
    // per-pair embedding projections and pair adjoints
    size_t fu, gfu, ue, edge_g, gp, q0, gEi;
    // weight-gradient scratch
    size_t gA_atom, gB_atom, zpart, wpart;
    // tensor-core modes: operand copies for the GEMMs
    size_t wbf, nbf, eu_bf, h1_bf, h2_bf, ga3_bf, ga2_bf, ga1_bf, gfu_bf;
    int64_t wbf_bytes;
    // per layer: the last radial-MLP layer's weight [3F][2F] and bias [3F]
    // with rows in plane-major order p*F + c (the blob keeps c*3 + p)
    size_t w3p;
    // tabulated radial functions (radial_table > 0)
    size_t tab, tab_tmp, dist;
    int64_t wpart_floats, zsplits;
    // MD
    size_t md_row_ptr, md_col, md_npairs, md_forces, md_energy, md_pos_ref, md_step, md_need, md_rebuilds;
    size_t total;
    int64_t node9;  // floats of one [9N][F] buffer
    int64_t cells;  // cell capacity
    int64_t maxU;   // undirected-edge capacity
};

}  // namespace tnet

namespace tnet {
// Host-side count of kernels enqueued by the library (all contexts).
void count_launch();

// Stages timed by the optional CUDA-event profiler (tnet_profile).
// Tuning knobs: 0 SIMT-GEMM CTAs per SM, 1 tcgen05 column tile for N = 3F,
// 2 tcgen05 column tile for N = 2F, 3 row-kernel blocks per SM, 4 pair-kernel
// blocks (256 threads) per SM, 5 programmatic dependent launch on (1) or off,
// 6 message-kernel form, 7 CTAs per cluster of the one-class tcgen05 GEMMs.
enum TuneKnob {
    T_GEMM_CTAS = 0, T_TC_BN_3F, T_TC_BN_2F, T_ROW_BLOCKS, T_PAIR_BLOCKS, T_PDL, T_MSG_KERNEL, T_TC_CLUSTER, T_NKNOBS
};

enum ProfTag {
    P_NBR = 0, P_PREP, P_EMB_EDGE, P_EMB_NODE, P_MLP1, P_MLP2, P_MLP3, P_MESSAGE, P_NODE_MIX,
    P_NODE_ELEM, P_OUTPUT, P_OUT_BWD, P_NODE_BWD, P_MSG_BWD, P_MLP_ELEM_BWD, P_MLP3_BWD, P_MLP2_BWD,
    P_MLP1_BWD, P_EMB_NODE_BWD, P_EMB_EDGE_BWD, P_FORCES, P_NTAGS
};
}  // namespace tnet

struct tnet_ctx {
    tnet_model_desc d;
    int max_atoms, max_systems;
    int64_t max_pairs;
    char *ws;
    size_t ws_bytes;
    tnet::Layout lay;
    tnet::RadialParams rp;
    int device, num_sms;
    // tuning knobs (tnet_set_tuning); see kTuneCandidates in api.cu
    int tune[8];
    // optional stage profiler
    int prof_on, prof_n, prof_cap;
    cudaEvent_t *prof_ev;
    int *prof_tag;
    // radial_table > 0: the tables hold the radial functions of the weights
    // last passed to tnet_radial_tables
    int tab_ready;
    // CUDA graph cache for tnet_md_step
    cudaGraphExec_t md_exec;
    const void *md_key[8];
    int64_t md_keyi[6];
    float md_keyf[3];
};

namespace tnet {
// Sequential stage markers: mark(tag) closes the open stage and opens the
// next one; CUDA events are recorded only when profiling is on and the
// stream is not being captured.
struct ProfSeq {
    tnet_ctx *c;
    cudaStream_t st;
    int slot;
    bool active;
    ProfSeq(tnet_ctx *ctx, cudaStream_t s);
    void mark(int tag);
    ~ProfSeq() { mark(-1); }
};
// Row-sum reductions for weight gradients (grad.cu).  Up to 3 classes of
// rows (blockIdx.z), e.g. the I, A and S coordinate planes.
struct WgradShape {
    int M, N;                 // output [M][N] per class
    int64_t rows[3];          // rows per class (capacity if rows_dev is set)
    int64_t row0[3];          // first row of each class in A and B
    const int32_t *rows_dev;  // optional device row count (class 0 only), times rows_mul
    int rows_mul;
    const float *A;           // A[row][m]
    int64_t lda;
    const float *B;           // B[row][n]
    int64_t ldb;
    int nclass;
};
// out[z][m][n] (+)= sum_rows A[r][m] B[r][n].  perm_f > 0: A's M = 3 perm_f
// columns are plane-major (m = p perm_f + c); out row c*3 + p receives row m.
int wgrad_outer(const WgradShape &P, float *partial, int64_t partial_cap, float *out, int accumulate, int sms,
                cudaStream_t st, int perm_f = 0);
// out[z][m] (+)= sum_rows A[r][m] * roww[r] (roww may be NULL); perm_f as above
int wgrad_colsum(const WgradShape &P, const float *roww, float *partial, int64_t partial_cap, float *out,
                 int accumulate, int sms, cudaStream_t st, int perm_f = 0);
int wgrad_layernorm(const float *gy, const float *x, const float2 *stats, int R, int C, float *partial,
                    int64_t partial_cap, float *out_g, int sms, cudaStream_t st);

int build_layout(const tnet_model_desc *d, int N, int S, int64_t E, Layout *L);
int validate_desc(const tnet_model_desc *d);
template <class T>
__host__ inline T *wsp(tnet_ctx *c, size_t off) {
    return reinterpret_cast<T *>(c->ws + off);
}
// gate: optional device flag; when it reads 0 every kernel of the call
// returns at once (a rebuild that the graph enqueues but the step skips)
int scan_exclusive_i32(const int32_t *in, int32_t *out, int n, int32_t *tmp, int32_t *total_dev,
                       int64_t *total64_dev, cudaStream_t st, const int32_t *gate = nullptr);
int tnet_kernel_setup(tnet_ctx *c);
int sys_bounds(const int32_t *batch, int N, int S, int32_t *sys_start, int32_t *sys_end,
               int32_t *status, cudaStream_t st);
int64_t weight_offsets(const tnet_model_desc *d, const float *base, struct Weights *w);
int neighbors_impl(tnet_ctx *ctx, int n_atoms, int n_systems, const float *pos, const int32_t *batch,
                   const float *box, float cutoff, int32_t *row_ptr, int32_t *col, int64_t cap,
                   int64_t *n_pairs_dev, int32_t *status_dev, cudaStream_t st, const int32_t *gate = nullptr);
int energy_forces_impl(tnet_ctx *ctx, const float *w, int n_atoms, int n_systems, const int32_t *z,
                       const float *pos, const int32_t *batch, const float *box,
                       const int32_t *row_ptr, const int32_t *col, const float *seed,
                       double *energy, float *forces, float *grad_w, int32_t *status_dev,
                       cudaStream_t st);
int radial_tables_impl(tnet_ctx *ctx, const float *w, cudaStream_t st);
int md_impl(tnet_ctx *ctx, const float *w, int n_atoms, const int32_t *z, const float *inv_mass,
            float *pos, float *vel, const float *box, float dt, float skin, int rebuild_every,
            int n_steps, double *e_kin, double *e_pot, int32_t *status_dev, cudaStream_t st);
}  // namespace tnet
