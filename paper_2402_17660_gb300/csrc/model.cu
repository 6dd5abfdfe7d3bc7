// TensorNet energy and forces (Sec. 2.1.1; Sec. 2 Fig. 1): forward pass and a
// hand-written reverse pass for the forces, on the compact I/A/S coordinates
// of internal.cuh.  FP32 arithmetic, FP64 per-system energy reduction.
//
// Pass structure (one call of tnet_energy_forces):
//   graph prep   reverse-edge index; undirected active-edge list (i < j,
//                d < cutoff) so the radial MLP runs once per pair (its output
//                depends only on d, hence g_ij = g_ji)
//   embedding    edge kernel (pair embedding x radial projections x edge
//                basis, segmented over CSR rows) -> per-atom norm/LayerNorm,
//                scalar MLP and channel mixing
//   L layers     normalise, mix, radial MLP per pair, message gather, tensor
//                products Y M + M Y, normalise, mix, residual X + dX + dX^2
//   output       I/A/S norms, LayerNorm, MLP head, FP64 sum per system
//   reverse      the adjoint of every step in reverse order, ending in one
//                3-vector dE/dr_ij per directed edge; forces are assembled
//                per atom from its row and the reverse edges (no atomics).
#include "gemm.cuh"
#include "internal.cuh"
#include "tc_gemm.cuh"

namespace tnet {

constexpr int kMU = 4;  // edges whose loads are in flight together in the row kernels
constexpr int kChunk = 128;  // row edges whose indices are staged in shared memory at a time

// ----------------------------------------------------------- weights ---
struct LayerW {
    const float *mlp1_w, *mlp1_b, *mlp2_w, *mlp2_b, *mlp3_w, *mlp3_b, *mix1_w, *mix2_w;
};
struct Weights {
    const float *emb, *emb2_w, *emb2_b, *dproj_w, *dproj_b, *emb_ln_g, *emb_ln_b, *emb_mlp1_w,
        *emb_mlp1_b, *emb_mlp2_w, *emb_mlp2_b, *emb_mix_w;
    LayerW layer[8];
    const float *out_ln_g, *out_ln_b, *out_w, *out_b, *head1_w, *head1_b, *head2_w, *head2_b;
};

// Offsets of the blob layout documented in tnet.h.  Returns the total.
int64_t weight_offsets(const tnet_model_desc *d, const float *base, Weights *w) {
    const int64_t F = d->F, K = d->K, Z = d->max_z;
    int64_t o = 0;
    auto take = [&](int64_t n) { const float *p = base ? base + o : nullptr; o += n; return p; };
    Weights t{};
    t.emb = take(Z * F);
    t.emb2_w = take(F * 2 * F); t.emb2_b = take(F);
    t.dproj_w = take(3 * F * K); t.dproj_b = take(3 * F);
    t.emb_ln_g = take(F); t.emb_ln_b = take(F);
    t.emb_mlp1_w = take(2 * F * F); t.emb_mlp1_b = take(2 * F);
    t.emb_mlp2_w = take(3 * F * 2 * F); t.emb_mlp2_b = take(3 * F);
    t.emb_mix_w = take(3 * F * F);
    for (int l = 0; l < d->L; ++l) {
        LayerW &L = t.layer[l];
        L.mlp1_w = take(F * K); L.mlp1_b = take(F);
        L.mlp2_w = take(2 * F * F); L.mlp2_b = take(2 * F);
        L.mlp3_w = take(3 * F * 2 * F); L.mlp3_b = take(3 * F);
        L.mix1_w = take(3 * F * F);
        L.mix2_w = take(3 * F * F);
    }
    t.out_ln_g = take(3 * F); t.out_ln_b = take(3 * F);
    t.out_w = take(F * 3 * F); t.out_b = take(F);
    t.head1_w = take(F / 2 * F); t.head1_b = take(F / 2);
    t.head2_w = take(F / 2); t.head2_b = take(1);
    if (w) *w = t;
    return o;
}

// --------------------------------------------------------- utilities ---
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over the block (blockDim.x a multiple of 32, <= 1024); all threads get it
__device__ __forceinline__ float block_sum(float v, float *sm) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sm[wid] = v;
    __syncthreads();
    float t = 0.f;
    for (int k = 0; k < nw; ++k) t += sm[k];
    return t;
}

// pair vector r_ij = mic(r_i - r_j) for rectangular or triclinic
// (lower-triangular) boxes, with fixed rounding (see mic_lower)
__device__ __forceinline__ void pair_vec(const float *__restrict__ pos, const float *__restrict__ box,
                                         const int32_t *__restrict__ batch, int i, int j, float &x,
                                         float &y, float &zz) {
    x = __fsub_rn(pos[3LL * i], pos[3LL * j]);
    y = __fsub_rn(pos[3LL * i + 1], pos[3LL * j + 1]);
    zz = __fsub_rn(pos[3LL * i + 2], pos[3LL * j + 2]);
    if (box) mic_box(x, y, zz, box + 9LL * (batch ? batch[i] : 0));
}

// ------------------------------------------------------- graph prep ---
// rev[e] = position of (j, i) in row j; one warp per row.
__global__ void k_rev(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int N,
                      int32_t *__restrict__ rev, int32_t *status) {
    pdl_entry();
    const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (i >= N) return;
    const int lane = threadIdx.x & 31;
    const int e0 = row_ptr[i];
    for (int e = e0 + lane; e < row_ptr[i + 1]; e += 32) {
        const int j = col[e];
        if (j < 0 || j >= N || (e > e0 && col[e - 1] >= j)) {  // rows must ascend strictly
            set_status(status, TNET_ERR_ARG);
            rev[e] = e;
            continue;
        }
        int lo = row_ptr[j], hi = row_ptr[j + 1];
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (col[mid] < i) lo = mid + 1;
            else hi = mid;
        }
        if (lo < row_ptr[j + 1] && col[lo] == i) rev[e] = lo;
        else {
            set_status(status, TNET_ERR_ARG);  // pair list not symmetric
            rev[e] = e;
        }
    }
}

// Upper (j > i) edges with d < rc, counted per row.
__global__ void k_upper_count(const float *__restrict__ pos, const float *__restrict__ box,
                              const int32_t *__restrict__ batch, const int32_t *__restrict__ row_ptr,
                              const int32_t *__restrict__ col, int N, float rc,
                              int32_t *__restrict__ ucnt) {
    pdl_entry();
    const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (i >= N) return;
    const int lane = threadIdx.x & 31;
    int cnt = 0;
    for (int e0 = row_ptr[i]; e0 < row_ptr[i + 1]; e0 += 32) {
        const int e = e0 + lane;
        bool up = false;
        if (e < row_ptr[i + 1]) {
            const int j = col[e];
            if (j > i && j < N) {
                float x, y, zz;
                pair_vec(pos, box, batch, i, j, x, y, zz);
                up = sqrtf(norm2_rn(x, y, zz)) < rc;
            }
        }
        cnt += __popc(__ballot_sync(0xffffffffu, up));
    }
    if (lane == 0) ucnt[i] = cnt;
}

__global__ void k_upper_assign(const float *__restrict__ pos, const float *__restrict__ box,
                               const int32_t *__restrict__ batch, const int32_t *__restrict__ row_ptr,
                               const int32_t *__restrict__ col, int N, float rc,
                               const int32_t *__restrict__ uoff, int32_t *__restrict__ pair_of,
                               int2 *__restrict__ uij, int32_t *__restrict__ ue) {
    pdl_entry();
    const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (i >= N) return;
    const int lane = threadIdx.x & 31;
    int base = uoff[i];
    for (int e0 = row_ptr[i]; e0 < row_ptr[i + 1]; e0 += 32) {
        const int e = e0 + lane;
        bool up = false;
        int j = -1;
        if (e < row_ptr[i + 1]) {
            j = col[e];
            if (j > i && j < N) {
                float x, y, zz;
                pair_vec(pos, box, batch, i, j, x, y, zz);
                up = sqrtf(norm2_rn(x, y, zz)) < rc;
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, up);
        if (e < row_ptr[i + 1] && j > i) {
            if (up) {
                const int u = base + __popc(m & ((1u << lane) - 1u));
                pair_of[e] = u;
                uij[u] = make_int2(i, j);
                ue[u] = e;
            } else {
                pair_of[e] = -1;
            }
        }
        base += __popc(m);
    }
}

__global__ void k_lower_assign(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                               const int32_t *__restrict__ rev, int N, int32_t *__restrict__ pair_of) {
    pdl_entry();
    const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (i >= N) return;
    const int lane = threadIdx.x & 31;
    for (int e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += 32) {
        const int j = col[e];
        // rev[e] == e marks a column that is out of range or has no reverse
        // edge (status ARG is set): the edge stays inactive
        if (j <= i) pair_of[e] = (j == i || rev[e] == e) ? -1 : pair_of[rev[e]];
    }
}

// Radial basis and cutoff of each undirected active edge, and its geometry
// (unit vector u_ij for i < j, and phi) for the embedding kernels.
__global__ void k_edge_rbf(const float *__restrict__ pos, const float *__restrict__ box,
                           const int32_t *__restrict__ batch, const int2 *__restrict__ uij,
                           const int32_t *__restrict__ nu, int maxU, RadialParams rp,
                           float *__restrict__ eu, float *__restrict__ phiu, float4 *__restrict__ geo,
                           OpCopy eu_cp) {
    pdl_entry();
    // a block takes groups of P = blockDim.x (<= 256) pairs: one thread per
    // pair computes its geometry, then all threads evaluate the P x K basis
    // values from it (coalesced writes of eu)
    __shared__ float s_d[256], s_phi[256];
    const int U = *nu, K = rp.K;
    const int P = blockDim.x < 256 ? blockDim.x : 256;
    for (int64_t u0 = (int64_t)blockIdx.x * P; u0 < U; u0 += (int64_t)gridDim.x * P) {
        const int np = U - u0 < P ? (int)(U - u0) : P;
        if (threadIdx.x < np) {
            const int u = (int)u0 + threadIdx.x;
            const int2 p = uij[u];
            float x, y, zz;
            pair_vec(pos, box, batch, p.x, p.y, x, y, zz);
            const float d = sqrtf(norm2_rn(x, y, zz));
            const float phi = cutoff_phi(d, rp);
            s_d[threadIdx.x] = d;
            s_phi[threadIdx.x] = phi;
            phiu[u] = phi;
            const float inv = 1.0f / d;
            geo[u] = make_float4(x * inv, y * inv, zz * inv, phi);  // u_ij for i < j, and phi
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < np * K; idx += blockDim.x) {
            const int q = idx / K, k = idx % K;
            float e, de;
            expnorm_k(s_d[q], k, rp, s_phi[q], 0.f, e, de);
            const int64_t t = (u0 + q) * K + k;
            eu[t] = e;
            opcopy_store(eu_cp, t, e);
        }
        __syncthreads();
    }
}

// ------------------------------------------------ tabulated radial functions ---
// The radial projections f(d) and every layer's filter g(d) depend on the pair
// distance alone.  In table mode they are evaluated in FP64, with their
// d-derivatives (forward mode through the same layers), at the grid d_k = k h
// (k < n, h = rc/(n - 1)).  Each interval [d_k, d_k+1] stores the cubic
// Hermite polynomial p(s) = c0 + c1 s + c2 s^2 + c3 s^3, s = (d - d_k)/h, whose
// coefficients are formed in FP64 before rounding to FP32: the derivative
// p'(s)/h then carries no cancellation between neighbouring table values, and
// the forces are the derivatives of the interpolated energy.

struct RadialParams64 {
    double rc, rl, alpha, beta, mu0, dmu;
    int K;
};

__device__ __forceinline__ void silu64(double a, double &v, double &g) {
    const double sg = 1.0 / (1.0 + exp(-a));
    v = a * sg;
    g = sg * (1.0 + a * (1.0 - sg));
}

// basis e_q(d_k) (the cosine cutoff included), de_q/dd, phi(d_k), dphi/dd
__global__ void k_tab_rbf(int n, double h, RadialParams64 rp, double *__restrict__ e, double *__restrict__ de,
                          double *__restrict__ phi, double *__restrict__ dphi) {
    pdl_entry();
    const int K = rp.K;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)n * K;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(t / K), q = (int)(t % K);
        const double d = k * h;
        const double ph = d < rp.rc ? 0.5 * (cospi(d / rp.rc) + 1.0) : 0.0;
        const double dph = d < rp.rc ? -0.5 * 3.141592653589793 / rp.rc * sinpi(d / rp.rc) : 0.0;
        const double ex = exp(rp.alpha * (rp.rl - d));
        const double u = ex - (rp.mu0 + q * rp.dmu);
        const double rho = exp(-rp.beta * u * u);
        e[t] = ph * rho;
        de[t] = dph * rho + ph * rho * (2.0 * rp.beta * u * rp.alpha * ex);
        if (q == 0) {
            phi[k] = ph;
            dphi[k] = dph;
        }
    }
}

// One dense layer of the radial chain at the grid points, FP64, with its
// tangent: a = x W^T + b, ta = tx W^T, and
//   mode 0 (hidden layers): y = silu(a),       ty = silu'(a) ta
//   mode 1 (projections f): y = a,             ty = ta
//   mode 2 (filters g):     y = phi silu(a),   ty = dphi silu(a) + phi silu'(a) ta
// 64 x 64 output tiles, 256 threads with 4 x 4 outputs (and tangents) each.
__global__ void __launch_bounds__(256)
    k_tab_layer(int n, int Nout, int Kin, const double *__restrict__ x, const double *__restrict__ tx,
                const float *__restrict__ Wt, const float *__restrict__ b, int mode, const double *__restrict__ phi,
                const double *__restrict__ dphi, double *__restrict__ y, double *__restrict__ ty) {
    pdl_entry();
    constexpr int T = 64, BK = 16;
    __shared__ double xs[BK][T], ts[BK][T], ws[BK][T];
    const int tid = threadIdx.x, tr = tid / 16, tc = tid % 16;
    const int m0 = blockIdx.y * T, n0 = blockIdx.x * T;
    double acc[4][4], tac[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = tac[i][j] = 0.0;
    for (int k0 = 0; k0 < Kin; k0 += BK) {
        for (int i = tid; i < BK * T; i += blockDim.x) {
            const int r = i / BK, kk = i % BK, gk = k0 + kk;
            const int gm = m0 + r, gn = n0 + r;
            const bool okx = gm < n && gk < Kin, okw = gn < Nout && gk < Kin;
            xs[kk][r] = okx ? x[(int64_t)gm * Kin + gk] : 0.0;
            ts[kk][r] = okx ? tx[(int64_t)gm * Kin + gk] : 0.0;
            ws[kk][r] = okw ? (double)Wt[(int64_t)gn * Kin + gk] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            double xv[4], tv[4], wv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                xv[i] = xs[kk][tr * 4 + i];
                tv[i] = ts[kk][tr * 4 + i];
                wv[i] = ws[kk][tc * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j] = fma(xv[i], wv[j], acc[i][j]);
                    tac[i][j] = fma(tv[i], wv[j], tac[i][j]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + tr * 4 + i;
        if (gm >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tc * 4 + j;
            if (gn >= Nout) continue;
            const double a = acc[i][j] + (double)b[gn], ta = tac[i][j];
            double v, g, out, tout;
            if (mode == 1) {
                out = a;
                tout = ta;
            } else {
                silu64(a, v, g);
                if (mode == 0) {
                    out = v;
                    tout = g * ta;
                } else {
                    out = phi[gm] * v;
                    tout = dphi[gm] * v + phi[gm] * g * ta;
                }
            }
            y[(int64_t)gm * Nout + gn] = out;
            ty[(int64_t)gm * Nout + gn] = tout;
        }
    }
}

// Hermite coefficients of each interval, [n-1][W] float4 (c0, c1, c2, c3):
//   c0 = v0, c1 = h v0', c2 = 3 (v1 - v0) - 2 h v0' - h v1', c3 = 2 (v0 - v1) + h v0' + h v1'
__global__ void k_tab_coef(int n, int W, double h, const double *__restrict__ v, const double *__restrict__ dv,
                           float4 *__restrict__ coef) {
    pdl_entry();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)(n - 1) * W;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / W;
        const int w = (int)(t % W);
        const double v0 = v[k * W + w], v1 = v[(k + 1) * W + w];
        const double d0 = h * dv[k * W + w], d1 = h * dv[(k + 1) * W + w];
        coef[k * W + w] = make_float4((float)v0, (float)d0, (float)(3.0 * (v1 - v0) - 2.0 * d0 - d1),
                                      (float)(2.0 * (v0 - v1) + d0 + d1));
    }
}

// A table-mode view of one radial function: the consumers (embedding,
// messages and their adjoints) evaluate p(s) and p'(s)/h of the pair's
// interval themselves, reading one float4 per channel (L2-resident tables).
struct TabFn {
    const float4 *coef;  // [n-1][3F]
    const float *dist;   // [U] pair distances
    int n;
    float inv_h;
};
__device__ __forceinline__ void tab_locate(const TabFn &T, int u, int &k, float &s) {
    const float x = T.dist[u] * T.inv_h;
    int kk = (int)floorf(x);
    kk = kk < 0 ? 0 : (kk > T.n - 2 ? T.n - 2 : kk);
    k = kk;
    s = x - (float)kk;
}
__device__ __forceinline__ float tab_value(const float4 &c, float s) {
    return fmaf(s, fmaf(s, fmaf(s, c.w, c.z), c.y), c.x);
}
__device__ __forceinline__ float tab_slope(const float4 &c, float s, float inv_h) {
    return fmaf(s, fmaf(s, 3.f * c.w, 2.f * c.z), c.y) * inv_h;
}

// per undirected pair: u_ij, phi (geo), phi alone (phiu) and d (dist)
__global__ void k_pair_geo(const float *__restrict__ pos, const float *__restrict__ box,
                           const int32_t *__restrict__ batch, const int2 *__restrict__ uij,
                           const int32_t *__restrict__ nu, RadialParams rp, float *__restrict__ phiu,
                           float4 *__restrict__ geo, float *__restrict__ dist) {
    pdl_entry();
    const int U = *nu;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < U; u += gridDim.x * blockDim.x) {
        const int2 p = uij[u];
        float x, y, zz;
        pair_vec(pos, box, batch, p.x, p.y, x, y, zz);
        const float d = sqrtf(norm2_rn(x, y, zz));
        const float phi = cutoff_phi(d, rp);
        const float inv = 1.0f / d;
        phiu[u] = phi;
        dist[u] = d;
        geo[u] = make_float4(x * inv, y * inv, zz * inv, phi);
    }
}

// Per-element pair-embedding tables: Ta[z] = W_e[:, :F] emb[z],
// Tb[z] = W_e[:, F:] emb[z] + b_e, so that Z_ij = Ta[z_i] + Tb[z_j].
__global__ void k_elem_tables(const float *__restrict__ emb, const float *__restrict__ W,
                              const float *__restrict__ b, int F, float *__restrict__ Ta,
                              float *__restrict__ Tb) {
    pdl_entry();
    // block per element z; warp per output row of W (lanes along the row, so
    // the reads of W are coalesced), a fixed-order warp reduction
    extern __shared__ float e[];
    const int z = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = threadIdx.x; k < F; k += blockDim.x) e[k] = emb[(int64_t)z * F + k];
    __syncthreads();
    for (int r = warp; r < 2 * F; r += nw) {  // rows c (Ta) and F + c (Tb)
        const int c = r % F, half = r / F;
        const float *w = W + (int64_t)c * 2 * F + half * F;
        float s = 0.f;
        for (int k = lane; k < F; k += 32) s = fmaf(w[k], e[k], s);
        s = warp_sum(s);
        if (lane == 0) {
            if (half == 0) Ta[(int64_t)z * F + c] = s;
            else Tb[(int64_t)z * F + c] = s + b[c];
        }
    }
}

// ------------------------------------------------------- embedding ---

struct EdgeGeo {
    int j, active;
    float d, u[3], phi, dphi;
};

__device__ __forceinline__ EdgeGeo edge_geo(const float *__restrict__ pos, const float *__restrict__ box,
                                            const int32_t *__restrict__ batch, int i, int j,
                                            const RadialParams &rp) {
    EdgeGeo g;
    g.j = j;
    float x, y, zz;
    pair_vec(pos, box, batch, i, j, x, y, zz);
    g.d = sqrtf(norm2_rn(x, y, zz));
    g.active = (g.d < rp.rc) && (g.d > 0.f);
    const float inv = g.d > 0.f ? 1.0f / g.d : 0.f;
    g.u[0] = x * inv; g.u[1] = y * inv; g.u[2] = zz * inv;
    g.phi = g.active ? cutoff_phi(g.d, rp) : 0.f;
    g.dphi = g.active ? cutoff_dphi(g.d, rp) : 0.f;
    return g;
}

// X_raw_i = sum_j phi Z_ij (f^I I0 + f^A A0(u) + f^S S0(u)) over the active
// edges of row i, in row order.  f^p = W^p e(d) + b^p depends only on d, so
// it is computed once per undirected pair by a GEMM (fu, columns p*F + c),
// or, with TAB, evaluated here from the Hermite table; u and phi come once
// per pair from geo (k_edge_rbf or k_pair_geo).
// Block = F threads (thread = channel), persistent over atoms; loads for kMU
// edges are in flight together.
template <int F, bool TAB>
__global__ void __launch_bounds__(F) k_emb_edges(const float4 *__restrict__ geo, const int32_t *__restrict__ z,
                                                 const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                                 const int32_t *__restrict__ pair_of, int N, int max_z,
                                                 const float *__restrict__ fu, TabFn tf, const float *__restrict__ Ta,
                                                 const float *__restrict__ Tb, float *__restrict__ Xraw,
                                                 int32_t *status, OpCopy Xraw_cp) {
    pdl_entry();
    __shared__ int32_t s_u[kChunk], s_zs[kChunk];  // pair index; element of the column atom, signed by direction
    __shared__ int32_t s_kt[TAB ? kChunk : 1];      // table mode: interval and offset of the pair distance
    __shared__ float s_st[TAB ? kChunk : 1];
    const int c = threadIdx.x;
    for (int i = blockIdx.x; i < N; i += gridDim.x) {
        int zi = z[i];
        if (zi < 0 || zi >= max_z) {
            set_status(status, TNET_ERR_Z);
            zi = 0;
        }
        const float ta = Ta[(int64_t)zi * F + c];
        float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const int e0 = row_ptr[i], e1 = row_ptr[i + 1];
        for (int cb = e0; cb < e1; cb += kChunk) {
            const int n = e1 - cb < kChunk ? e1 - cb : kChunk;
            __syncthreads();
            for (int t = c; t < n; t += F) {
                const int u = pair_of[cb + t];
                s_u[t] = u;
                int zj = 0, j = i;
                if (u >= 0) {
                    j = col[cb + t];
                    zj = z[j];
                    zj = (zj < 0 || zj >= max_z) ? 0 : zj;
                }
                s_zs[t] = j > i ? zj : -1 - zj;   // u_ij = +u of the pair when i is its first atom
                if constexpr (TAB) {
                    int kt = 0;
                    float st = 0.f;
                    if (u >= 0) tab_locate(tf, u, kt, st);
                    s_kt[t] = kt;
                    s_st[t] = st;
                }
            }
            __syncthreads();
            for (int k0 = 0; k0 < n; k0 += kMU) {
                int uu[kMU], zz[kMU];
#pragma unroll
                for (int k = 0; k < kMU; ++k) {
                    uu[k] = k0 + k < n ? s_u[k0 + k] : -1;
                    zz[k] = k0 + k < n ? s_zs[k0 + k] : 0;
                }
                float f[kMU][3], tb[kMU];
                float4 gk[kMU];
#pragma unroll
                for (int k = 0; k < kMU; ++k) {
                    if (uu[k] < 0) continue;
                    if constexpr (TAB) {
                        const float4 *cp = tf.coef + (int64_t)s_kt[k0 + k] * 3 * F + c;
                        const float st = s_st[k0 + k];
                        f[k][0] = tab_value(cp[0], st); f[k][1] = tab_value(cp[F], st); f[k][2] = tab_value(cp[2 * F], st);
                    } else {
                        const float *fp = fu + (int64_t)uu[k] * 3 * F + c;
                        f[k][0] = fp[0]; f[k][1] = fp[F]; f[k][2] = fp[2 * F];
                    }
                    tb[k] = Tb[(int64_t)(zz[k] >= 0 ? zz[k] : -1 - zz[k]) * F + c];
                    gk[k] = geo[uu[k]];
                }
#pragma unroll
                for (int k = 0; k < kMU; ++k) {
                    if (uu[k] < 0) continue;
                    const float sg = zz[k] >= 0 ? 1.0f : -1.0f;
                    const float ux = sg * gk[k].x, uy = sg * gk[k].y, uz = sg * gk[k].z;
                    const float pz = gk[k].w * (ta + tb[k]);
                    const float cI = pz * f[k][0], cA = pz * f[k][1], cS = pz * f[k][2];
                    v[0] += cI;
                    v[1] += cA * ux; v[2] += cA * uy; v[3] += cA * uz;
                    v[4] += cS * (ux * ux - (1.0f / 3.0f));
                    v[5] += cS * (uy * uy - (1.0f / 3.0f));
                    v[6] += cS * ux * uy; v[7] += cS * ux * uz; v[8] += cS * uy * uz;
                }
            }
        }
        store_coords(Xraw, i, c, N, F, v);
        store_coords_cp(Xraw_cp, i, c, N, F, v);
    }
}

// q0 = ||X_raw|| per channel, LayerNorm over channels -> n0; caches (mean, rstd)
__global__ void k_norm_ln(const float *__restrict__ X, int N, int F, const float *__restrict__ g,
                          const float *__restrict__ b, float *__restrict__ n0, float2 *__restrict__ ln,
                          float *__restrict__ q0) {
    pdl_entry();
    __shared__ float sm[32];
    const int i = blockIdx.x, c = threadIdx.x;
    float v[9];
    load_coords(X, i, c, N, F, v);
    const float q = cnorm(v);
    const float mean = block_sum(q, sm) / F;
    const float dv = q - mean;
    const float var = block_sum(dv * dv, sm) / F;
    const float rstd = rsqrtf(var + 1e-5f);
    n0[(int64_t)i * F + c] = dv * rstd * g[c] + b[c];
    q0[(int64_t)i * F + c] = q;
    if (c == 0) ln[i] = make_float2(mean, rstd);
}

// X0 = s_p * U (p = class of the coordinate), s channel-major [N][F][3]
__global__ void k_emb_scale(const float *__restrict__ U, const float *__restrict__ s, int N, int F,
                            float *__restrict__ X0) {
    pdl_entry();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)N * F;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / F), c = (int)(t % F);
        float v[9];
        load_coords(U, i, c, N, F, v);
        const float *si = s + ((int64_t)i * F + c) * 3;
        v[0] *= si[0];
#pragma unroll
        for (int k = 1; k < 4; ++k) v[k] *= si[1];
#pragma unroll
        for (int k = 4; k < 9; ++k) v[k] *= si[2];
        store_coords(X0, i, c, N, F, v);
    }
}

// ----------------------------------------------------- interaction ---
// Xn = X / (||X|| + 1)
__global__ void k_node_norm(const float *__restrict__ X, int N, int F, float *__restrict__ qn,
                            float *__restrict__ Xn, OpCopy Xn_cp) {
    pdl_entry();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)N * F;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / F), c = (int)(t % F);
        float v[9];
        load_coords(X, i, c, N, F, v);
        const float q = cnorm(v);
        qn[t] = q;
        const float r = 1.0f / (q + 1.0f);
#pragma unroll
        for (int k = 0; k < 9; ++k) v[k] *= r;
        store_coords(Xn, i, c, N, F, v);
        store_coords_cp(Xn_cp, i, c, N, F, v);
    }
}

// M_i = sum_j g^p_ij Y^p_j over the row (block = F threads, thread = channel).
// The filter is never stored: g = phi(d) SiLU(a3) is formed here from the last
// radial layer's pre-activation a3 of pair u, stored plane-major, a3[u][p][c],
// so each of its three loads is one coalesced F-channel row, and phi of the
// pair (the same expression as the GEMM epilogue would evaluate).  The row's pair and column indices are staged in
// shared memory (one coalesced load per chunk of kChunk edges), so each group of
// kMU edges waits for one round of gathers, not for its indices first; the
// sums still run in row order.  F is a template parameter so the coordinate
// offsets are immediates.
//
// RB consecutive rows per block, one group of F threads per row (named
// barrier 1 + group): consecutive atoms share most of their neighbours (the
// three atoms of a water, the next molecule of the lattice), so the groups of
// a block gather mostly the same rows of Y at about the same time (columns
// ascend in every row) and the repeats hit the SM's L1 instead of L2.
template <int F, bool TAB, int RB>
__global__ void __launch_bounds__(F * RB, (768 / (F * RB)) > 0 ? 768 / (F * RB) : 1)
    k_message(const int32_t *__restrict__ row_ptr,
                                                    const int32_t *__restrict__ col,
                                                    const int32_t *__restrict__ pair_of, const float *__restrict__ a3,
                                                    const float *__restrict__ phiu, TabFn tg,
                                                    const float *__restrict__ Y, int N, float *__restrict__ M) {
    pdl_entry();
    __shared__ int32_t s_u_all[RB][kChunk], s_j_all[RB][kChunk];
    __shared__ int32_t s_kt_all[RB][TAB ? kChunk : 1];
    __shared__ float s_st_all[RB][TAB ? kChunk : 1];
    const int grp = RB > 1 ? (int)threadIdx.x / F : 0, c = RB > 1 ? (int)threadIdx.x % F : (int)threadIdx.x;
    int32_t *s_u = s_u_all[grp], *s_j = s_j_all[grp], *s_kt = s_kt_all[grp];
    float *s_st = s_st_all[grp];
    for (int i = blockIdx.x * RB + grp; i < N; i += gridDim.x * RB) {
        float m[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const int e0 = row_ptr[i], e1 = row_ptr[i + 1];
        for (int cb = e0; cb < e1; cb += kChunk) {
            const int n = e1 - cb < kChunk ? e1 - cb : kChunk;
            group_sync<F, RB>(grp);  // the previous chunk is consumed
            for (int t = c; t < n; t += F) {
                const int u = pair_of[cb + t];
                s_u[t] = u;
                s_j[t] = col[cb + t];
                if constexpr (TAB) {
                    int kt = 0;
                    float st = 0.f;
                    if (u >= 0) tab_locate(tg, u, kt, st);
                    s_kt[t] = kt;
                    s_st[t] = st;
                }
            }
            group_sync<F, RB>(grp);
            for (int k0 = 0; k0 < n; k0 += kMU) {
                int uu[kMU], jj[kMU];
#pragma unroll
                for (int k = 0; k < kMU; ++k) {
                    uu[k] = k0 + k < n ? s_u[k0 + k] : -1;
                    jj[k] = k0 + k < n ? s_j[k0 + k] : 0;
                }
                float g[kMU][3], y[kMU][9], ph[kMU];
#pragma unroll
                for (int k = 0; k < kMU; ++k) {
                    if (uu[k] < 0) continue;
                    if constexpr (TAB) {
                        const float4 *cp = tg.coef + (int64_t)s_kt[k0 + k] * 3 * F + c;
                        const float st = s_st[k0 + k];
                        g[k][0] = tab_value(cp[0], st); g[k][1] = tab_value(cp[F], st); g[k][2] = tab_value(cp[2 * F], st);
                    } else {
                        const float *ap = a3 + (int64_t)uu[k] * 3 * F + c;
                        g[k][0] = ap[0]; g[k][1] = ap[F]; g[k][2] = ap[2 * F];
                        ph[k] = phiu[uu[k]];
                    }
                    load_coords(Y, jj[k], c, N, F, y[k]);
                }
#pragma unroll
                for (int k = 0; k < kMU; ++k) {
                    if (uu[k] < 0) continue;
                    if constexpr (!TAB) {
#pragma unroll
                        for (int p = 0; p < 3; ++p) g[k][p] = silu_f(g[k][p]) * ph[k];
                    }
                    m[0] = fmaf(g[k][0], y[k][0], m[0]);
#pragma unroll
                    for (int q = 1; q < 4; ++q) m[q] = fmaf(g[k][1], y[k][q], m[q]);
#pragma unroll
                    for (int q = 4; q < 9; ++q) m[q] = fmaf(g[k][2], y[k][q], m[q]);
                }
            }
        }
        store_coords(M, i, c, N, F, m);
    }
}

// T = Y M + M Y; Tn = decomp(T) / (||T|| + 1)
__global__ void k_node_update(const float *__restrict__ Y, const float *__restrict__ M, int N, int F,
                              float *__restrict__ Tn, OpCopy Tn_cp) {
    pdl_entry();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)N * F;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / F), c = (int)(t % F);
        float yv[9], mv[9], Yf[9], Mf[9], A[9], B[9], T[9], tc[9];
        load_coords(Y, i, c, N, F, yv);
        load_coords(M, i, c, N, F, mv);
        expand(yv, Yf);
        expand(mv, Mf);
        mm3(Yf, Mf, A);
        mm3(Mf, Yf, B);
#pragma unroll
        for (int k = 0; k < 9; ++k) T[k] = A[k] + B[k];
        decomp(T, tc);
        const float r = 1.0f / (cnorm(tc) + 1.0f);
#pragma unroll
        for (int k = 0; k < 9; ++k) tc[k] *= r;
        store_coords(Tn, i, c, N, F, tc);
        store_coords_cp(Tn_cp, i, c, N, F, tc);
    }
}

// X_out = Xn + dX + dX dX
__global__ void k_residual(const float *__restrict__ Xn, const float *__restrict__ dX, int N, int F,
                           float *__restrict__ Xout) {
    pdl_entry();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)N * F;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / F), c = (int)(t % F);
        float xv[9], dv[9], Q[9], Q2[9], q2[9];
        load_coords(Xn, i, c, N, F, xv);
        load_coords(dX, i, c, N, F, dv);
        expand(dv, Q);
        mm3(Q, Q, Q2);
        decomp(Q2, q2);
#pragma unroll
        for (int k = 0; k < 9; ++k) xv[k] += dv[k] + q2[k];
        store_coords(Xout, i, c, N, F, xv);
    }
}

// ---------------------------------------------------------- output ---
// h = (||I||, ||A||, ||S||) in blocks of F, LayerNorm over 3F
__global__ void k_out_norms(const float *__restrict__ X, int N, int F, const float *__restrict__ g,
                            const float *__restrict__ b, float *__restrict__ h, float *__restrict__ hn,
                            float2 *__restrict__ ln) {
    pdl_entry();
    __shared__ float sm[32];
    const int i = blockIdx.x, c = threadIdx.x;
    float v[9];
    load_coords(X, i, c, N, F, v);
    const float sxx = v[4], syy = v[5], szz = -(v[4] + v[5]);
    const float hv[3] = {3.0f * v[0] * v[0], 2.0f * (v[1] * v[1] + v[2] * v[2] + v[3] * v[3]),
                         sxx * sxx + syy * syy + szz * szz + 2.0f * (v[6] * v[6] + v[7] * v[7] + v[8] * v[8])};
    const float mean = block_sum(hv[0] + hv[1] + hv[2], sm) / (3 * F);
    const float d0 = hv[0] - mean, d1 = hv[1] - mean, d2 = hv[2] - mean;
    const float var = block_sum(d0 * d0 + d1 * d1 + d2 * d2, sm) / (3 * F);
    const float rstd = rsqrtf(var + 1e-5f);
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const int64_t o = (int64_t)i * 3 * F + p * F + c;
        h[o] = hv[p];
        hn[o] = (hv[p] - mean) * rstd * g[p * F + c] + b[p * F + c];
    }
    if (c == 0) ln[i] = make_float2(mean, rstd);
}

// E_i = w2 . t_i + b2 (one warp per atom)
__global__ void k_head(const float *__restrict__ t, int N, int H, const float *__restrict__ w2,
                       const float *__restrict__ b2, float *__restrict__ Ei) {
    pdl_entry();
    const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (i >= N) return;
    const int lane = threadIdx.x & 31;
    float s = 0.f;
    for (int k = lane; k < H; k += 32) s = fmaf(t[(int64_t)i * H + k], w2[k], s);
    s = warp_sum(s);
    if (lane == 0) Ei[i] = s + b2[0];
}

// E_s = sum of E_i over the system, in FP64 (one block per system)
__global__ void k_energy(const float *__restrict__ Ei, const int32_t *__restrict__ sys_start,
                         const int32_t *__restrict__ sys_end, double *__restrict__ energy) {
    pdl_entry();
    __shared__ double sm[32];
    const int s = blockIdx.x;
    double acc = 0.0;
    for (int n = sys_start[s] + threadIdx.x; n < sys_end[s]; n += blockDim.x) acc += (double)Ei[n];
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
        energy[s] = t;
    }
}

// ========================================================= reverse ===
__global__ void k_head_bwd(const float *__restrict__ at, int N, int H, const float *__restrict__ w2,
                           const float *__restrict__ seed, const int32_t *__restrict__ batch,
                           float *__restrict__ gat) {
    pdl_entry();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)N * H;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / H), k = (int)(t % H);
        const float gE = seed ? seed[batch ? batch[i] : 0] : 1.0f;
        gat[t] = gE * w2[k] * silu_grad_f(at[t]);
    }
}

// LayerNorm backward over 3F, then d(norms)/d(coordinates) -> gX
__global__ void k_out_norms_bwd(const float *__restrict__ X, const float *__restrict__ h,
                                const float *__restrict__ ghn, const float2 *__restrict__ ln,
                                const float *__restrict__ g, int N, int F, float *__restrict__ gX) {
    pdl_entry();
    __shared__ float sm[32];
    const int i = blockIdx.x, c = threadIdx.x;
    const float2 mr = ln[i];
    float xh[3], gx[3];
    float s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const int64_t o = (int64_t)i * 3 * F + p * F + c;
        xh[p] = (h[o] - mr.x) * mr.y;
        gx[p] = ghn[o] * g[p * F + c];
        s1 += gx[p];
        s2 += gx[p] * xh[p];
    }
    const float m1 = block_sum(s1, sm) / (3 * F);
    const float m2 = block_sum(s2, sm) / (3 * F);
    float gh[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) gh[p] = mr.y * (gx[p] - m1 - xh[p] * m2);
    float v[9], gv[9];
    load_coords(X, i, c, N, F, v);
    gv[0] = 6.0f * v[0] * gh[0];
#pragma unroll
    for (int k = 1; k < 4; ++k) gv[k] = 4.0f * v[k] * gh[1];
    gv[4] = (4.0f * v[4] + 2.0f * v[5]) * gh[2];
    gv[5] = (4.0f * v[5] + 2.0f * v[4]) * gh[2];
#pragma unroll
    for (int k = 6; k < 9; ++k) gv[k] = 4.0f * v[k] * gh[2];
    store_coords(gX, i, c, N, F, gv);
}

// X_out = Xn + dX + dX dX:  g_dX = g + expand^T(G Q^T + Q^T G), G = decomp^T(g)
__global__ void k_residual_bwd(const float *__restrict__ gX, const float *__restrict__ dX, int N, int F,
                               float *__restrict__ gdX, OpCopy gdX_cp) {
    pdl_entry();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)N * F;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / F), c = (int)(t % F);
        float g[9], dv[9], G[9], Q[9], A[9], B[9], GQ[9], gq[9];
        load_coords(gX, i, c, N, F, g);
        load_coords(dX, i, c, N, F, dv);
        decomp_T(g, G);
        expand(dv, Q);
        mm3_nt(G, Q, A);
        mm3_tn(Q, G, B);
#pragma unroll
        for (int k = 0; k < 9; ++k) GQ[k] = A[k] + B[k];
        expand_T(GQ, gq);
#pragma unroll
        for (int k = 0; k < 9; ++k) g[k] += gq[k];
        store_coords(gdX, i, c, N, F, g);
        store_coords_cp(gdX_cp, i, c, N, F, g);
    }
}

// Tn = decomp(Y M + M Y) / (p + 1): gradients to Y (written) and M (written)
__global__ void k_T_bwd(const float *__restrict__ Y, const float *__restrict__ M,
                        const float *__restrict__ gTn, int N, int F, float *__restrict__ gY,
                        float *__restrict__ gM) {
    pdl_entry();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)N * F;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / F), c = (int)(t % F);
        float yv[9], mv[9], Yf[9], Mf[9], A[9], B[9], T[9], tc[9], g[9], ng[9], GT[9];
        load_coords(Y, i, c, N, F, yv);
        load_coords(M, i, c, N, F, mv);
        load_coords(gTn, i, c, N, F, g);
        expand(yv, Yf);
        expand(mv, Mf);
        mm3(Yf, Mf, A);
        mm3(Mf, Yf, B);
#pragma unroll
        for (int k = 0; k < 9; ++k) T[k] = A[k] + B[k];
        decomp(T, tc);
        const float den = cnorm(tc) + 1.0f;
        float dot = 0.f;
#pragma unroll
        for (int k = 0; k < 9; ++k) dot = fmaf(g[k], tc[k], dot);
        cnorm_grad(tc, ng);
        const float a = 1.0f / den, bcoef = dot / (den * den);
#pragma unroll
        for (int k = 0; k < 9; ++k) g[k] = g[k] * a - bcoef * ng[k];
        decomp_T(g, GT);
        // dY = G M^T + M^T G ; dM = Y^T G + G Y^T
        float gYf[9], gMf[9], out[9];
        mm3_nt(GT, Mf, A);
        mm3_tn(Mf, GT, B);
#pragma unroll
        for (int k = 0; k < 9; ++k) gYf[k] = A[k] + B[k];
        mm3_tn(Yf, GT, A);
        mm3_nt(GT, Yf, B);
#pragma unroll
        for (int k = 0; k < 9; ++k) gMf[k] = A[k] + B[k];
        expand_T(gYf, out);
        store_coords(gY, i, c, N, F, out);
        expand_T(gMf, out);
        store_coords(gM, i, c, N, F, out);
    }
}

// Message adjoint and the last radial layer's elementwise adjoint.  For atom
// i (block, thread per channel):
//   gY_i += sum_j g^p_ij gM_j                          (g_ij = g_ji)
//   gg^p[u(i,j)] = <gM_i, Y^p_j> + <gM_j, Y^p_i>        for upper edges j > i
// with g = phi silu(a3) formed here from the pair's stored a3 and phi (the
// filter itself is never stored), and, for the same upper edge:
//   ga3 = gg phi silu'(a3)       (fp32 if ga3 != NULL, plus its operand copy)
//   gphi[u] += sum over the 3F entries of gg silu(a3)
// Each undirected pair is handled once, by its upper edge: no atomics.  The
// gphi sum is reduced per warp, then over the warps in a fixed order at the end
// of each chunk.  Rows ascend, so the upper edges are the row's suffix: the
// lower part gathers gM_j alone (kMU edges in flight), the upper part gM_j,
// Y_j and a3 together (kMUU edges).  Indices are staged in shared memory as in
// k_message; the gY sums run in row order.
// With TAB (tabulated radial functions) g and dg/dd come from the table: the
// kernel adds sum dE/dg dg/dd to gphi (then dE/dd of the pair) and writes no
// dE/da3.
// RB consecutive rows per block, one group of F threads per row, as in
// k_message (the groups' repeated gathers of gM_j and Y_j hit L1).
constexpr int kMUU = 2;
template <int F, bool TAB, int RB>
__global__ void __launch_bounds__(F * RB, (512 / (F * RB)) > 0 ? 512 / (F * RB) : 1)
    k_message_bwd(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                  const int32_t *__restrict__ pair_of, const float *__restrict__ Y,
                  const float *__restrict__ gM, const float *__restrict__ a3, const float *__restrict__ phiu,
                  TabFn tg, int N, float *__restrict__ gY, OpCopy gY_cp, float *__restrict__ ga3, OpCopy ga3_cp,
                  float *__restrict__ gphi) {
    pdl_entry();
    constexpr int NW = F / 32;
    constexpr int CH = RB >= 4 ? kChunk / 2 : kChunk;  // staged edges per chunk (static smem stays below 48 KB)
    __shared__ int32_t s_u_all[RB][CH], s_j_all[RB][CH];
    __shared__ int32_t s_kt_all[RB][TAB ? CH : 1];
    __shared__ float s_st_all[RB][TAB ? CH : 1];
    __shared__ float s_red_all[RB][CH][NW];
    __shared__ float s_yi_all[RB][9][F], s_gmi_all[RB][9][F];  // row i's Y and gM (per thread's channel)
    const int grp = RB > 1 ? (int)threadIdx.x / F : 0, c = RB > 1 ? (int)threadIdx.x % F : (int)threadIdx.x;
    const int lane = c & 31, warp = c >> 5;
    int32_t *s_u = s_u_all[grp], *s_j = s_j_all[grp], *s_kt = s_kt_all[grp];
    float *s_st = s_st_all[grp];
    float(*s_red)[NW] = s_red_all[grp];
    float(*s_yi)[F] = s_yi_all[grp];
    float(*s_gmi)[F] = s_gmi_all[grp];
    for (int i = blockIdx.x * RB + grp; i < N; i += gridDim.x * RB) {
        float acc[9];
        {
            float t[9];
            load_coords(Y, i, c, N, F, t);
#pragma unroll
            for (int q = 0; q < 9; ++q) s_yi[q][c] = t[q];
            load_coords(gM, i, c, N, F, t);
#pragma unroll
            for (int q = 0; q < 9; ++q) s_gmi[q][c] = t[q];
        }
        load_coords(gY, i, c, N, F, acc);
        const int e0 = row_ptr[i], e1 = row_ptr[i + 1];
        int eu = e0, hi = e1;  // eu = first edge with col > i
        while (eu < hi) {
            const int mid = (eu + hi) >> 1;
            if (col[mid] <= i) eu = mid + 1;
            else hi = mid;
        }
        for (int cb = e0; cb < e1; cb += CH) {
            const int n = e1 - cb < CH ? e1 - cb : CH;
            group_sync<F, RB>(grp);
            for (int t = c; t < n; t += F) {
                const int u = pair_of[cb + t];
                s_u[t] = u;
                s_j[t] = col[cb + t];
                if constexpr (TAB) {
                    int kt = 0;
                    float st = 0.f;
                    if (u >= 0) tab_locate(tg, u, kt, st);
                    s_kt[t] = kt;
                    s_st[t] = st;
                }
            }
            group_sync<F, RB>(grp);
            const int nl = eu - cb < 0 ? 0 : (eu - cb < n ? eu - cb : n);  // lower edges of the chunk
            for (int k0 = 0; k0 < nl; k0 += kMU) {
                int uu[kMU], jj[kMU];
#pragma unroll
                for (int k = 0; k < kMU; ++k) {
                    uu[k] = k0 + k < nl ? s_u[k0 + k] : -1;
                    jj[k] = k0 + k < nl ? s_j[k0 + k] : 0;
                }
                float g[kMU][3], gmj[kMU][9], ph[kMU];
#pragma unroll
                for (int k = 0; k < kMU; ++k) {
                    if (uu[k] < 0) continue;
                    if constexpr (TAB) {
                        const float4 *cp = tg.coef + (int64_t)s_kt[k0 + k] * 3 * F + c;
                        const float st = s_st[k0 + k];
                        g[k][0] = tab_value(cp[0], st); g[k][1] = tab_value(cp[F], st); g[k][2] = tab_value(cp[2 * F], st);
                    } else {
                        const float *ap = a3 + (int64_t)uu[k] * 3 * F + c;
                        g[k][0] = ap[0]; g[k][1] = ap[F]; g[k][2] = ap[2 * F];
                        ph[k] = phiu[uu[k]];
                    }
                    load_coords(gM, jj[k], c, N, F, gmj[k]);
                }
#pragma unroll
                for (int k = 0; k < kMU; ++k) {
                    if (uu[k] < 0) continue;
                    if constexpr (!TAB) {
#pragma unroll
                        for (int p = 0; p < 3; ++p) g[k][p] = silu_f(g[k][p]) * ph[k];
                    }
                    acc[0] = fmaf(g[k][0], gmj[k][0], acc[0]);
#pragma unroll
                    for (int q = 1; q < 4; ++q) acc[q] = fmaf(g[k][1], gmj[k][q], acc[q]);
#pragma unroll
                    for (int q = 4; q < 9; ++q) acc[q] = fmaf(g[k][2], gmj[k][q], acc[q]);
                }
            }
            for (int k0 = nl; k0 < n; k0 += kMUU) {
                int uu[kMUU], jj[kMUU];
#pragma unroll
                for (int k = 0; k < kMUU; ++k) {
                    uu[k] = k0 + k < n ? s_u[k0 + k] : -1;
                    jj[k] = k0 + k < n ? s_j[k0 + k] : 0;
                }
                float g[kMUU][3], gmj[kMUU][9], yj[kMUU][9], a[kMUU][3], phi[kMUU];
#pragma unroll
                for (int k = 0; k < kMUU; ++k) {
                    if (uu[k] < 0) continue;
                    if constexpr (TAB) {   // g and dg/dd (in a) from the pair's interval
                        const float4 *cp = tg.coef + (int64_t)s_kt[k0 + k] * 3 * F + c;
                        const float st = s_st[k0 + k];
#pragma unroll
                        for (int p = 0; p < 3; ++p) {
                            const float4 cq = cp[p * F];
                            g[k][p] = tab_value(cq, st);
                            a[k][p] = tab_slope(cq, st, tg.inv_h);
                        }
                        phi[k] = 0.f;
                    } else {
                        const int64_t o = (int64_t)uu[k] * 3 * F + c;
                        a[k][0] = a3[o]; a[k][1] = a3[o + F]; a[k][2] = a3[o + 2 * F];
                        phi[k] = phiu[uu[k]];
#pragma unroll
                        for (int p = 0; p < 3; ++p) g[k][p] = silu_f(a[k][p]) * phi[k];
                    }
                    load_coords(gM, jj[k], c, N, F, gmj[k]);
                    load_coords(Y, jj[k], c, N, F, yj[k]);
                }
#pragma unroll
                for (int k = 0; k < kMUU; ++k) {
                    if (uu[k] < 0) continue;
                    acc[0] = fmaf(g[k][0], gmj[k][0], acc[0]);
#pragma unroll
                    for (int q = 1; q < 4; ++q) acc[q] = fmaf(g[k][1], gmj[k][q], acc[q]);
#pragma unroll
                    for (int q = 4; q < 9; ++q) acc[q] = fmaf(g[k][2], gmj[k][q], acc[q]);
                    float sp[3];
                    sp[0] = s_gmi[0][c] * yj[k][0] + gmj[k][0] * s_yi[0][c];
                    sp[1] = 0.f; sp[2] = 0.f;
#pragma unroll
                    for (int q = 1; q < 4; ++q) sp[1] += s_gmi[q][c] * yj[k][q] + gmj[k][q] * s_yi[q][c];
#pragma unroll
                    for (int q = 4; q < 9; ++q) sp[2] += s_gmi[q][c] * yj[k][q] + gmj[k][q] * s_yi[q][c];
                    const int64_t o = (int64_t)uu[k] * 3 * F + c;
                    float r = 0.f;
#pragma unroll
                    for (int p = 0; p < 3; ++p) {
                        if constexpr (TAB) {
                            r = fmaf(sp[p], a[k][p], r);
                        } else {
                            float sv, sd;
                            silu_and_grad_f(a[k][p], sv, sd);
                            r = fmaf(sp[p], sv, r);
                            const float ga = sp[p] * phi[k] * sd;
                            if (ga3) ga3[o + p * F] = ga;
                            opcopy_store(ga3_cp, o + p * F, ga);
                        }
                    }
                    r = warp_sum(r);
                    if (lane == 0) s_red[k0 + k - nl][warp] = r;
                }
            }
            group_sync<F, RB>(grp);
            for (int t = c; t < n - nl; t += F) {
                const int u = s_u[nl + t];
                if (u < 0) continue;
                float r = 0.f;
#pragma unroll
                for (int w = 0; w < NW; ++w) r += s_red[t][w];
                gphi[u] += r;
            }
        }
        store_coords(gY, i, c, N, F, acc);
        store_coords_cp(gY_cp, i, c, N, F, acc);
    }
}

// ------------------------------------------- warp-per-row message kernels ---
// The same sums as k_message and k_message_bwd (exact mode), with one warp per
// row and four consecutive channels per lane: every gathered row of F floats
// is one float4 load per lane (F / 128 of them), so the load, address and
// index instructions per edge fall by four against a thread per channel, the
// dE/dphi sum of a pair is one warp reduction (no shared-memory partials or
// block barriers), and each warp keeps two edges' gathers in flight.  Built
// for F = 128 (the adjoint's per-warp staging of row i is 9 KB).  Offsets are
// 32-bit (the host checks 9 N F < 2^31).
constexpr int kV4Warps = 4;  // warps (rows in flight) per block

__device__ __forceinline__ float4 ld4(const float *__restrict__ p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *__restrict__ p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ void fma4(float4 &a, float s, const float4 &x) {
    a.x = fmaf(s, x.x, a.x); a.y = fmaf(s, x.y, a.y); a.z = fmaf(s, x.z, a.z); a.w = fmaf(s, x.w, a.w);
}
__device__ __forceinline__ void fma4v(float4 &a, const float4 &s, const float4 &x) {
    a.x = fmaf(s.x, x.x, a.x); a.y = fmaf(s.y, x.y, a.y); a.z = fmaf(s.z, x.z, a.z); a.w = fmaf(s.w, x.w, a.w);
}
// first element (in floats) of coordinate row q (0..8) of atom n in a node
// tensor laid out as I rows [0, N), A rows [N, 4N), S rows [4N, 9N)
__device__ __forceinline__ uint32_t coord_row(int q, uint32_t n, uint32_t N, uint32_t F) {
    return (q == 0 ? n : (q < 4 ? N + 3u * n + (uint32_t)(q - 1) : 4u * N + 5u * n + (uint32_t)(q - 4))) * F;
}
// plane p (I, A, S) of coordinate q
__device__ __forceinline__ constexpr int plane_of(int q) { return q == 0 ? 0 : (q < 4 ? 1 : 2); }

template <int F>
__global__ void __launch_bounds__(32 * kV4Warps, 3) k_message_v4(const int32_t *__restrict__ row_ptr,
                                                              const int32_t *__restrict__ col,
                                                              const int32_t *__restrict__ pair_of,
                                                              const float *__restrict__ a3,
                                                              const float *__restrict__ phiu,
                                                              const float *__restrict__ Y, int N,
                                                              float *__restrict__ M) {
    pdl_entry();
    static_assert(F % 128 == 0, "four channels per lane");
    constexpr int PER = F / 128;  // float4 per lane per row
    constexpr int KM = 2;         // edges in flight per warp
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * kV4Warps;
    for (int i = blockIdx.x * kV4Warps + (threadIdx.x >> 5); i < N; i += nw) {
        float4 m[9][PER];
#pragma unroll
        for (int q = 0; q < 9; ++q)
#pragma unroll
            for (int r = 0; r < PER; ++r) m[q][r] = make_float4(0.f, 0.f, 0.f, 0.f);
        const int e0 = row_ptr[i], e1 = row_ptr[i + 1];
        for (int eb = e0; eb < e1; eb += 32) {
            const int n = e1 - eb < 32 ? e1 - eb : 32;
            int u_l = -1, j_l = 0;
            float ph_l = 0.f;
            if (lane < n) {
                u_l = pair_of[eb + lane];
                j_l = col[eb + lane];
                if (u_l >= 0) ph_l = phiu[u_l];
            }
            for (int k0 = 0; k0 < n; k0 += KM) {
                int uu[KM], jj[KM];
                float ph[KM];
#pragma unroll
                for (int k = 0; k < KM; ++k) {
                    const int src = k0 + k < n ? k0 + k : 0;
                    uu[k] = __shfl_sync(0xffffffffu, u_l, src);
                    jj[k] = __shfl_sync(0xffffffffu, j_l, src);
                    ph[k] = __shfl_sync(0xffffffffu, ph_l, src);
                    if (k0 + k >= n) uu[k] = -1;
                }
                float4 g[KM][3][PER], y[KM][9][PER];
#pragma unroll
                for (int k = 0; k < KM; ++k) {
                    if (uu[k] < 0) continue;
                    const uint32_t ab = (uint32_t)uu[k] * 3u * F + 4u * lane;
#pragma unroll
                    for (int p = 0; p < 3; ++p)
#pragma unroll
                        for (int r = 0; r < PER; ++r) g[k][p][r] = ld4(a3 + ab + p * F + 128 * r);
#pragma unroll
                    for (int q = 0; q < 9; ++q) {
                        const uint32_t yb = coord_row(q, (uint32_t)jj[k], (uint32_t)N, F) + 4u * lane;
#pragma unroll
                        for (int r = 0; r < PER; ++r) y[k][q][r] = ld4(Y + yb + 128 * r);
                    }
                }
#pragma unroll
                for (int k = 0; k < KM; ++k) {
                    if (uu[k] < 0) continue;
#pragma unroll
                    for (int p = 0; p < 3; ++p)
#pragma unroll
                        for (int r = 0; r < PER; ++r) {
                            float4 &v = g[k][p][r];
                            v.x = silu_f(v.x) * ph[k]; v.y = silu_f(v.y) * ph[k];
                            v.z = silu_f(v.z) * ph[k]; v.w = silu_f(v.w) * ph[k];
                        }
#pragma unroll
                    for (int q = 0; q < 9; ++q)
#pragma unroll
                        for (int r = 0; r < PER; ++r) fma4v(m[q][r], g[k][plane_of(q)][r], y[k][q][r]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const uint32_t mb = coord_row(q, (uint32_t)i, (uint32_t)N, F) + 4u * lane;
#pragma unroll
            for (int r = 0; r < PER; ++r) st4(M + mb + 128 * r, m[q][r]);
        }
    }
}

// Adjoint, warp per row: gY_i += sum_j g_ij gM_j over the row; for the upper
// edges (j > i) also dE/dg of the pair, dE/da3 = dE/dg phi SiLU'(a3) and
// dE/dphi += sum dE/dg SiLU(a3) (one warp reduction, in the lane order).
// Row i's own Y and gM sit in shared memory (per warp) for the upper edges'
// dot products.  One lower edge's gathers are in flight at a time, and an
// upper edge gathers gM_j (with a3) and then Y_j, which keeps the kernel
// within 255 registers without spills (two blocks, eight warps per SM).
template <int F, int MINB>
__global__ void __launch_bounds__(32 * kV4Warps, MINB)
    k_message_bwd_v4(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                     const int32_t *__restrict__ pair_of, const float *__restrict__ Y,
                     const float *__restrict__ gM, const float *__restrict__ a3, const float *__restrict__ phiu,
                     int N, float *__restrict__ gY, OpCopy gY_cp, float *__restrict__ ga3, OpCopy ga3_cp,
                     float *__restrict__ gphi) {
    pdl_entry();
    static_assert(F % 128 == 0, "four channels per lane");
    constexpr int PER = F / 128;
    constexpr int KM = 1;   // lower edges in flight per warp
    __shared__ float4 s_own[kV4Warps][2][9][F / 4];  // row i's Y and gM
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float4(*s_y)[F / 4] = s_own[w][0];
    float4(*s_gm)[F / 4] = s_own[w][1];
    const int nw = gridDim.x * kV4Warps;
    for (int i = blockIdx.x * kV4Warps + w; i < N; i += nw) {
        // row i's Y and gM into shared memory, one coordinate row at a time
#pragma unroll 1
        for (int q = 0; q < 9; ++q) {
            const uint32_t b = coord_row(q, (uint32_t)i, (uint32_t)N, F) + 4u * lane;
#pragma unroll
            for (int r = 0; r < PER; ++r) {
                s_y[q][lane + 32 * r] = ld4(Y + b + 128 * r);
                s_gm[q][lane + 32 * r] = ld4(gM + b + 128 * r);
            }
        }
        float4 acc[9][PER];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const uint32_t b = coord_row(q, (uint32_t)i, (uint32_t)N, F) + 4u * lane;
#pragma unroll
            for (int r = 0; r < PER; ++r) acc[q][r] = ld4(gY + b + 128 * r);
        }
        // each lane reads back only what it wrote: no barrier needed
        const int e0 = row_ptr[i], e1 = row_ptr[i + 1];
        int eu = e0, hi = e1;  // first edge with col > i
        while (eu < hi) {
            const int mid = (eu + hi) >> 1;
            if (col[mid] <= i) eu = mid + 1;
            else hi = mid;
        }
        for (int eb = e0; eb < e1; eb += 32) {
            const int n = e1 - eb < 32 ? e1 - eb : 32;
            int u_l = -1, j_l = 0;
            float ph_l = 0.f;
            if (lane < n) {
                u_l = pair_of[eb + lane];
                j_l = col[eb + lane];
                if (u_l >= 0) ph_l = phiu[u_l];
            }
            const int nl = eu - eb < 0 ? 0 : (eu - eb < n ? eu - eb : n);  // lower edges of the batch
            for (int k0 = 0; k0 < nl; k0 += KM) {
                int uu[KM], jj[KM];
                float ph[KM];
#pragma unroll
                for (int k = 0; k < KM; ++k) {
                    const int src = k0 + k < nl ? k0 + k : 0;
                    uu[k] = __shfl_sync(0xffffffffu, u_l, src);
                    jj[k] = __shfl_sync(0xffffffffu, j_l, src);
                    ph[k] = __shfl_sync(0xffffffffu, ph_l, src);
                    if (k0 + k >= nl) uu[k] = -1;
                }
                float4 g[KM][3][PER], gm[KM][9][PER];
#pragma unroll
                for (int k = 0; k < KM; ++k) {
                    if (uu[k] < 0) continue;
                    const uint32_t ab = (uint32_t)uu[k] * 3u * F + 4u * lane;
#pragma unroll
                    for (int p = 0; p < 3; ++p)
#pragma unroll
                        for (int r = 0; r < PER; ++r) g[k][p][r] = ld4(a3 + ab + p * F + 128 * r);
#pragma unroll
                    for (int q = 0; q < 9; ++q) {
                        const uint32_t b = coord_row(q, (uint32_t)jj[k], (uint32_t)N, F) + 4u * lane;
#pragma unroll
                        for (int r = 0; r < PER; ++r) gm[k][q][r] = ld4(gM + b + 128 * r);
                    }
                }
#pragma unroll
                for (int k = 0; k < KM; ++k) {
                    if (uu[k] < 0) continue;
#pragma unroll
                    for (int p = 0; p < 3; ++p)
#pragma unroll
                        for (int r = 0; r < PER; ++r) {
                            float4 &v = g[k][p][r];
                            v.x = silu_f(v.x) * ph[k]; v.y = silu_f(v.y) * ph[k];
                            v.z = silu_f(v.z) * ph[k]; v.w = silu_f(v.w) * ph[k];
                        }
#pragma unroll
                    for (int q = 0; q < 9; ++q)
#pragma unroll
                        for (int r = 0; r < PER; ++r) fma4v(acc[q][r], g[k][plane_of(q)][r], gm[k][q][r]);
                }
            }
            for (int k = nl; k < n; ++k) {  // upper edges, one at a time
                const int u = __shfl_sync(0xffffffffu, u_l, k);
                const int j = __shfl_sync(0xffffffffu, j_l, k);
                const float ph = __shfl_sync(0xffffffffu, ph_l, k);
                if (u < 0) continue;
                // two rounds of gathers (gM_j with a3, then Y_j), so that only
                // one 9-row block is live at a time
                const uint32_t ab = (uint32_t)u * 3u * F + 4u * lane;
                float4 sp[3][PER], gv[3][PER];
                float rsum = 0.f;
                {
                    float4 a[3][PER], gm[9][PER];
#pragma unroll
                    for (int p = 0; p < 3; ++p)
#pragma unroll
                        for (int r = 0; r < PER; ++r) {
                            a[p][r] = ld4(a3 + ab + p * F + 128 * r);
                            sp[p][r] = make_float4(0.f, 0.f, 0.f, 0.f);
                        }
#pragma unroll
                    for (int q = 0; q < 9; ++q) {
                        const uint32_t bq = coord_row(q, (uint32_t)j, (uint32_t)N, F) + 4u * lane;
#pragma unroll
                        for (int r = 0; r < PER; ++r) gm[q][r] = ld4(gM + bq + 128 * r);
                    }
#pragma unroll
                    for (int p = 0; p < 3; ++p)
#pragma unroll
                        for (int r = 0; r < PER; ++r) {
                            const float4 v = a[p][r];
                            gv[p][r] = make_float4(silu_f(v.x) * ph, silu_f(v.y) * ph, silu_f(v.z) * ph,
                                                   silu_f(v.w) * ph);
                        }
#pragma unroll
                    for (int q = 0; q < 9; ++q)
#pragma unroll
                        for (int r = 0; r < PER; ++r) {
                            fma4v(acc[q][r], gv[plane_of(q)][r], gm[q][r]);
                            fma4v(sp[plane_of(q)][r], gm[q][r], s_y[q][lane + 32 * r]);
                        }
                }
                {
                    float4 yj[9][PER];
#pragma unroll
                    for (int q = 0; q < 9; ++q) {
                        const uint32_t bq = coord_row(q, (uint32_t)j, (uint32_t)N, F) + 4u * lane;
#pragma unroll
                        for (int r = 0; r < PER; ++r) yj[q][r] = ld4(Y + bq + 128 * r);
                    }
#pragma unroll
                    for (int q = 0; q < 9; ++q)
#pragma unroll
                        for (int r = 0; r < PER; ++r) fma4v(sp[plane_of(q)][r], s_gm[q][lane + 32 * r], yj[q][r]);
                }
#pragma unroll
                for (int p = 0; p < 3; ++p)
#pragma unroll
                    for (int r = 0; r < PER; ++r) {
                        // a3 again (just read by this warp: an L1 or L2 hit) rather
                        // than held through both gather rounds
                        const float4 ar = ld4(a3 + ab + p * F + 128 * r);
                        const float av[4] = {ar.x, ar.y, ar.z, ar.w};
                        const float sv4[4] = {sp[p][r].x, sp[p][r].y, sp[p][r].z, sp[p][r].w};
                        float gav[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            float sv, sd;
                            silu_and_grad_f(av[c], sv, sd);
                            rsum = fmaf(sv4[c], sv, rsum);
                            gav[c] = sv4[c] * ph * sd;
                        }
                        const uint32_t o = ab + p * F + 128 * r;
                        if (ga3) st4(ga3 + o, make_float4(gav[0], gav[1], gav[2], gav[3]));
                        if (ga3_cp.mode) {
                            opcopy_store(ga3_cp, o, gav[0]);
                            opcopy_store(ga3_cp, o + 1, gav[1]);
                            opcopy_store(ga3_cp, o + 2, gav[2]);
                            opcopy_store(ga3_cp, o + 3, gav[3]);
                        }
                    }
                rsum = warp_sum(rsum);
                if (lane == 0) gphi[u] += rsum;
            }
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const uint32_t b = coord_row(q, (uint32_t)i, (uint32_t)N, F) + 4u * lane;
#pragma unroll
            for (int r = 0; r < PER; ++r) {
                st4(gY + b + 128 * r, acc[q][r]);
                if (gY_cp.mode) {
                    opcopy_store(gY_cp, b + 128 * r, acc[q][r].x);
                    opcopy_store(gY_cp, b + 128 * r + 1, acc[q][r].y);
                    opcopy_store(gY_cp, b + 128 * r + 2, acc[q][r].z);
                    opcopy_store(gY_cp, b + 128 * r + 3, acc[q][r].w);
                }
            }
        }
    }
}

// Xn = X / (q + 1):  gX = gXn / (q + 1) - <gXn, X> / (q + 1)^2 * dq/dX (in place)
__global__ void k_node_norm_bwd(const float *__restrict__ X, const float *__restrict__ qn, int N, int F,
                                float *__restrict__ gX) {
    pdl_entry();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)N * F;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / F), c = (int)(t % F);
        float xv[9], g[9], ng[9];
        load_coords(X, i, c, N, F, xv);
        load_coords(gX, i, c, N, F, g);
        const float den = qn[t] + 1.0f;
        float dot = 0.f;
#pragma unroll
        for (int k = 0; k < 9; ++k) dot = fmaf(g[k], xv[k], dot);
        cnorm_grad(xv, ng);
        const float a = 1.0f / den, b = dot / (den * den);
#pragma unroll
        for (int k = 0; k < 9; ++k) g[k] = g[k] * a - b * ng[k];
        store_coords(gX, i, c, N, F, g);
    }
}

// X0 = s_p * U:  gU = s_p gX0; gas2 = <gX0, U>_p * silu'(as2)
__global__ void k_emb_scale_bwd(const float *__restrict__ gX0, const float *__restrict__ U,
                                const float *__restrict__ s, const float *__restrict__ as2, int N, int F,
                                float *__restrict__ gU, float *__restrict__ gas2, OpCopy gU_cp) {
    pdl_entry();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)N * F;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / F), c = (int)(t % F);
        float g[9], uv[9];
        load_coords(gX0, i, c, N, F, g);
        load_coords(U, i, c, N, F, uv);
        const float *si = s + t * 3;
        float gs[3] = {g[0] * uv[0], 0.f, 0.f};
#pragma unroll
        for (int k = 1; k < 4; ++k) gs[1] += g[k] * uv[k];
#pragma unroll
        for (int k = 4; k < 9; ++k) gs[2] += g[k] * uv[k];
        g[0] *= si[0];
#pragma unroll
        for (int k = 1; k < 4; ++k) g[k] *= si[1];
#pragma unroll
        for (int k = 4; k < 9; ++k) g[k] *= si[2];
        store_coords(gU, i, c, N, F, g);
        store_coords_cp(gU_cp, i, c, N, F, g);
#pragma unroll
        for (int p = 0; p < 3; ++p) gas2[t * 3 + p] = gs[p] * silu_grad_f(as2[t * 3 + p]);
    }
}

// LayerNorm of q0 = ||X_raw||: adds gq0 * dq0/dX_raw to gXraw (which holds the
// channel-mixing adjoint)
__global__ void k_ln0_bwd(const float *__restrict__ Xraw, const float *__restrict__ gn0,
                          const float2 *__restrict__ ln, const float *__restrict__ g, int N, int F,
                          float *__restrict__ gXraw) {
    pdl_entry();
    __shared__ float sm[32];
    const int i = blockIdx.x, c = threadIdx.x;
    float v[9], gv[9], ng[9];
    load_coords(Xraw, i, c, N, F, v);
    const float2 mr = ln[i];
    const float xh = (cnorm(v) - mr.x) * mr.y;
    const float gx = gn0[(int64_t)i * F + c] * g[c];
    const float m1 = block_sum(gx, sm) / F;
    const float m2 = block_sum(gx * xh, sm) / F;
    const float gq = mr.y * (gx - m1 - xh * m2);
    load_coords(gXraw, i, c, N, F, gv);
    cnorm_grad(v, ng);
#pragma unroll
    for (int k = 0; k < 9; ++k) gv[k] = fmaf(gq, ng[k], gv[k]);
    store_coords(gXraw, i, c, N, F, gv);
}

// Embedding edge adjoint, one warp per atom i (lane = channels lane + 32k).
// For each active directed edge e = (i, j) of the row it writes
//   edge_g[e] = (dE/dphi, dE/du) of that directed use of the pair (u = r_ij/d),
// and for upper edges (j > i) the pair's projection adjoint summed over both
// directions, gfu[u] = dE/df^p (columns p*F + c), which needs gXraw_j.
// With want_z it also sums the pair-embedding adjoints dE/dZ per atom as
// receiver (gA_atom) and as sender (gB_atom) for the embedding-table gradients.
template <int CPL>
__global__ void k_emb_bwd(const float *__restrict__ pos, const float *__restrict__ box,
                          const int32_t *__restrict__ batch, const int32_t *__restrict__ z,
                          const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                          const int32_t *__restrict__ pair_of, int N, int max_z, RadialParams rp,
                          const float *__restrict__ fu, const float *__restrict__ Ta,
                          const float *__restrict__ Tb, const float *__restrict__ gXraw, int want_z,
                          float *__restrict__ gfu, float4 *__restrict__ edge_g, float *__restrict__ gA_atom,
                          float *__restrict__ gB_atom, OpCopy gfu_cp) {
    pdl_entry();
    constexpr int F = CPL * 32;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t ii = warp0; ii < N; ii += nwarps) {
        const int i = (int)ii;
        int zi = z[i];
        zi = (zi < 0 || zi >= max_z) ? 0 : zi;
        float gi[CPL][9], ta[CPL], tbi[CPL], accA[CPL], accB[CPL];
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            const int c = lane + 32 * k;
            load_coords(gXraw, i, c, N, F, gi[k]);
            ta[k] = Ta[(int64_t)zi * F + c];
            tbi[k] = Tb[(int64_t)zi * F + c];
            accA[k] = accB[k] = 0.f;
        }
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int u = pair_of[e];
            if (u < 0) {
                if (lane == 0) edge_g[e] = make_float4(0.f, 0.f, 0.f, 0.f);
                continue;
            }
            const int j = col[e];
            float x, y, zz;
            pair_vec(pos, box, batch, i, j, x, y, zz);
            const float d = sqrtf(norm2_rn(x, y, zz));
            const float inv = 1.0f / d;
            const float ux = x * inv, uy = y * inv, uz = zz * inv;
            const float phi = cutoff_phi(d, rp);
            const float bxx = ux * ux - (1.0f / 3.0f), byy = uy * uy - (1.0f / 3.0f);
            const float bxy = ux * uy, bxz = ux * uz, byz = uy * uz;
            int zj = z[j];
            zj = (zj < 0 || zj >= max_z) ? 0 : zj;
            const bool upper = j > i;
            const bool need_j = upper || want_z;
            float gphi = 0.f, gux = 0.f, guy = 0.f, guz = 0.f;
#pragma unroll
            for (int k = 0; k < CPL; ++k) {
                const int c = lane + 32 * k;
                const float *fp = fu + (int64_t)u * 3 * F + c;
                const float f0 = fp[0], f1 = fp[F], f2 = fp[2 * F];
                const float Zij = ta[k] + Tb[(int64_t)zj * F + c];
                const float *g = gi[k];
                const float gc0 = g[0];
                const float gcA = g[1] * ux + g[2] * uy + g[3] * uz;
                const float gcS = g[4] * bxx + g[5] * byy + g[6] * bxy + g[7] * bxz + g[8] * byz;
                const float dot = gc0 * f0 + gcA * f1 + gcS * f2;
                gphi = fmaf(Zij, dot, gphi);
                const float cA = phi * Zij * f1, cS = phi * Zij * f2;
                gux += cA * g[1] + cS * (2.f * ux * g[4] + uy * g[6] + uz * g[7]);
                guy += cA * g[2] + cS * (2.f * uy * g[5] + ux * g[6] + uz * g[8]);
                guz += cA * g[3] + cS * (ux * g[7] + uy * g[8]);
                accA[k] = fmaf(phi, dot, accA[k]);
                if (need_j) {
                    float gj[9];
                    load_coords(gXraw, j, c, N, F, gj);
                    // the reverse use (j, i): u_ji = -u, the S basis is even in u
                    const float hc0 = gj[0];
                    const float hcA = -(gj[1] * ux + gj[2] * uy + gj[3] * uz);
                    const float hcS = gj[4] * bxx + gj[5] * byy + gj[6] * bxy + gj[7] * bxz + gj[8] * byz;
                    const float Zji = Ta[(int64_t)zj * F + c] + tbi[k];
                    if (upper) {
                        float *o = gfu + (int64_t)u * 3 * F + c;
                        const float o0 = phi * (Zij * gc0 + Zji * hc0);
                        const float o1 = phi * (Zij * gcA + Zji * hcA);
                        const float o2 = phi * (Zij * gcS + Zji * hcS);
                        o[0] = o0;
                        o[F] = o1;
                        o[2 * F] = o2;
                        const int64_t ob = (int64_t)u * 3 * F + c;
                        opcopy_store(gfu_cp, ob, o0);
                        opcopy_store(gfu_cp, ob + F, o1);
                        opcopy_store(gfu_cp, ob + 2 * F, o2);
                    }
                    accB[k] = fmaf(phi, hc0 * f0 + hcA * f1 + hcS * f2, accB[k]);
                }
            }
            gphi = warp_sum(gphi);
            gux = warp_sum(gux);
            guy = warp_sum(guy);
            guz = warp_sum(guz);
            if (lane == 0) edge_g[e] = make_float4(gphi, gux, guy, guz);
        }
        if (want_z) {
#pragma unroll
            for (int k = 0; k < CPL; ++k) {
                gA_atom[(int64_t)i * F + lane + 32 * k] = accA[k];
                gB_atom[(int64_t)i * F + lane + 32 * k] = accB[k];
            }
        }
    }
}

// Embedding edge adjoint for forces only, one warp per undirected pair
// (lane = channels lane + 32k): both directed uses of the pair at once,
//   edge_g[e]      = (dE/dphi, dE/du) of the use (i, j), u = r_ij / d
//   edge_g[rev e]  = the same for (j, i), u_ji = -u
//   gfu[u]         = dE/df^p summed over both uses (columns p*F + c).
// Pair-parallel, so small systems still fill the GPU.
template <int CPL, bool TAB>
__global__ void k_emb_bwd_pairs(const float4 *__restrict__ geo, const int32_t *__restrict__ z,
                                const int2 *__restrict__ uij, const int32_t *__restrict__ ue,
                                const int32_t *__restrict__ rev, const int32_t *__restrict__ nu, int N, int max_z,
                                const float *__restrict__ fu, TabFn tf, const float *__restrict__ Ta,
                                const float *__restrict__ Tb, const float *__restrict__ gXraw,
                                float *__restrict__ gfu, float4 *__restrict__ edge_g,
                                OpCopy gfu_cp, float *__restrict__ dEdd) {
    pdl_entry();
    constexpr int F = CPL * 32;
    const int lane = threadIdx.x & 31;
    const int U = *nu;
    for (int64_t uu = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; uu < U;
         uu += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int u = (int)uu;
        const int2 p = uij[u];
        const int i = p.x, j = p.y;
        const float4 gu = geo[u];  // u_ij and phi of the pair (k_edge_rbf or k_pair_geo)
        const float ux = gu.x, uy = gu.y, uz = gu.z, phi = gu.w;
        const float bxx = ux * ux - (1.0f / 3.0f), byy = uy * uy - (1.0f / 3.0f);
        const float bxy = ux * uy, bxz = ux * uz, byz = uy * uz;
        int zi = z[i], zj = z[j];
        zi = (zi < 0 || zi >= max_z) ? 0 : zi;
        zj = (zj < 0 || zj >= max_z) ? 0 : zj;
        float a_phi = 0.f, ax = 0.f, ay = 0.f, az = 0.f;   // use (i, j)
        float b_phi = 0.f, bx = 0.f, by = 0.f, bz = 0.f;   // use (j, i), gradient w.r.t. u_ji
        float gd = 0.f;                                    // sum dE/df df/dd (table mode)
        int kt = 0;
        float st = 0.f;
        if constexpr (TAB) tab_locate(tf, u, kt, st);
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            const int c = lane + 32 * k;
            float f0, f1, f2, df0 = 0.f, df1 = 0.f, df2 = 0.f;
            if constexpr (TAB) {
                const float4 *cp = tf.coef + (int64_t)kt * 3 * F + c;
                const float4 q0 = cp[0], q1 = cp[F], q2 = cp[2 * F];
                f0 = tab_value(q0, st); f1 = tab_value(q1, st); f2 = tab_value(q2, st);
                df0 = tab_slope(q0, st, tf.inv_h); df1 = tab_slope(q1, st, tf.inv_h); df2 = tab_slope(q2, st, tf.inv_h);
            } else {
                const float *fp = fu + (int64_t)u * 3 * F + c;
                f0 = fp[0]; f1 = fp[F]; f2 = fp[2 * F];
            }
            float gi[9], gj[9];
            load_coords(gXraw, i, c, N, F, gi);
            load_coords(gXraw, j, c, N, F, gj);
            const float Zij = Ta[(int64_t)zi * F + c] + Tb[(int64_t)zj * F + c];
            const float Zji = Ta[(int64_t)zj * F + c] + Tb[(int64_t)zi * F + c];
            // use (i, j)
            const float gc0 = gi[0];
            const float gcA = gi[1] * ux + gi[2] * uy + gi[3] * uz;
            const float gcS = gi[4] * bxx + gi[5] * byy + gi[6] * bxy + gi[7] * bxz + gi[8] * byz;
            a_phi = fmaf(Zij, gc0 * f0 + gcA * f1 + gcS * f2, a_phi);
            {
                const float cA = phi * Zij * f1, cS = phi * Zij * f2;
                ax += cA * gi[1] + cS * (2.f * ux * gi[4] + uy * gi[6] + uz * gi[7]);
                ay += cA * gi[2] + cS * (2.f * uy * gi[5] + ux * gi[6] + uz * gi[8]);
                az += cA * gi[3] + cS * (ux * gi[7] + uy * gi[8]);
            }
            // use (j, i): v = -u, the S basis is even in u
            const float vx = -ux, vy = -uy, vz = -uz;
            const float hc0 = gj[0];
            const float hcA = gj[1] * vx + gj[2] * vy + gj[3] * vz;
            const float hcS = gj[4] * bxx + gj[5] * byy + gj[6] * bxy + gj[7] * bxz + gj[8] * byz;
            b_phi = fmaf(Zji, hc0 * f0 + hcA * f1 + hcS * f2, b_phi);
            {
                const float cA = phi * Zji * f1, cS = phi * Zji * f2;
                bx += cA * gj[1] + cS * (2.f * vx * gj[4] + vy * gj[6] + vz * gj[7]);
                by += cA * gj[2] + cS * (2.f * vy * gj[5] + vx * gj[6] + vz * gj[8]);
                bz += cA * gj[3] + cS * (vx * gj[7] + vy * gj[8]);
            }
            const float o0 = phi * (Zij * gc0 + Zji * hc0);
            const float o1 = phi * (Zij * gcA + Zji * hcA);
            const float o2 = phi * (Zij * gcS + Zji * hcS);
            const int64_t ob = (int64_t)u * 3 * F + c;
            if constexpr (TAB) {   // no projection weights to go back through
                gd += o0 * df0 + o1 * df1 + o2 * df2;
            } else {
                gfu[ob] = o0;
                gfu[ob + F] = o1;
                gfu[ob + 2 * F] = o2;
                opcopy_store(gfu_cp, ob, o0);
                opcopy_store(gfu_cp, ob + F, o1);
                opcopy_store(gfu_cp, ob + 2 * F, o2);
            }
        }
        a_phi = warp_sum(a_phi); ax = warp_sum(ax); ay = warp_sum(ay); az = warp_sum(az);
        b_phi = warp_sum(b_phi); bx = warp_sum(bx); by = warp_sum(by); bz = warp_sum(bz);
        if constexpr (TAB) gd = warp_sum(gd);
        if (lane == 0) {
            if constexpr (TAB) dEdd[u] += gd;
            const int e = ue[u];
            edge_g[e] = make_float4(a_phi, ax, ay, az);
            edge_g[rev[e]] = make_float4(b_phi, bx, by, bz);
        }
    }
}

// The same adjoint with four consecutive channels per lane (F = 128, exact
// mode, forces only): every gathered row of gX_raw, the pair's projections
// and the element tables are float4 loads, a quarter of the load and address
// instructions of the strided form above.  Offsets are 32-bit (the host
// checks the sizes).
template <int F>
__global__ void __launch_bounds__(256) k_emb_bwd_pairs_v4(const float4 *__restrict__ geo,
                                                          const int32_t *__restrict__ z,
                                                          const int2 *__restrict__ uij, const int32_t *__restrict__ ue,
                                                          const int32_t *__restrict__ rev,
                                                          const int32_t *__restrict__ nu, int N, int max_z,
                                                          const float *__restrict__ fu, const float *__restrict__ Ta,
                                                          const float *__restrict__ Tb,
                                                          const float *__restrict__ gXraw, float *__restrict__ gfu,
                                                          float4 *__restrict__ edge_g, OpCopy gfu_cp) {
    pdl_entry();
    static_assert(F == 128, "one float4 per lane and row");
    const int lane = threadIdx.x & 31;
    const int U = *nu;
    const uint32_t c4 = 4u * lane;
    for (int64_t uu = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; uu < U;
         uu += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int u = (int)uu;
        const int2 p = uij[u];
        const int i = p.x, j = p.y;
        const float4 gu = geo[u];
        const float ux = gu.x, uy = gu.y, uz = gu.z, phi = gu.w;
        const float bxx = ux * ux - (1.0f / 3.0f), byy = uy * uy - (1.0f / 3.0f);
        const float bxy = ux * uy, bxz = ux * uz, byz = uy * uz;
        int zi = z[i], zj = z[j];
        zi = (zi < 0 || zi >= max_z) ? 0 : zi;
        zj = (zj < 0 || zj >= max_z) ? 0 : zj;
        const uint32_t fb = (uint32_t)u * 3u * F + c4;
        const float4 f0 = ld4(fu + fb), f1 = ld4(fu + fb + F), f2 = ld4(fu + fb + 2 * F);
        float4 gi[9], gj[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            gi[q] = ld4(gXraw + coord_row(q, (uint32_t)i, (uint32_t)N, F) + c4);
            gj[q] = ld4(gXraw + coord_row(q, (uint32_t)j, (uint32_t)N, F) + c4);
        }
        const float4 tai = ld4(Ta + (uint32_t)zi * F + c4), tbj = ld4(Tb + (uint32_t)zj * F + c4);
        const float4 taj = ld4(Ta + (uint32_t)zj * F + c4), tbi = ld4(Tb + (uint32_t)zi * F + c4);
        float a_phi = 0.f, ax = 0.f, ay = 0.f, az = 0.f;
        float b_phi = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
        const float vx = -ux, vy = -uy, vz = -uz;
        float o[3][4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            auto el = [k](const float4 &v) { return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w)); };
            float g[9], h[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                g[q] = el(gi[q]);
                h[q] = el(gj[q]);
            }
            const float F0 = el(f0), F1 = el(f1), F2 = el(f2);
            const float Zij = el(tai) + el(tbj), Zji = el(taj) + el(tbi);
            const float gc0 = g[0];
            const float gcA = g[1] * ux + g[2] * uy + g[3] * uz;
            const float gcS = g[4] * bxx + g[5] * byy + g[6] * bxy + g[7] * bxz + g[8] * byz;
            a_phi = fmaf(Zij, gc0 * F0 + gcA * F1 + gcS * F2, a_phi);
            {
                const float cA = phi * Zij * F1, cS = phi * Zij * F2;
                ax += cA * g[1] + cS * (2.f * ux * g[4] + uy * g[6] + uz * g[7]);
                ay += cA * g[2] + cS * (2.f * uy * g[5] + ux * g[6] + uz * g[8]);
                az += cA * g[3] + cS * (ux * g[7] + uy * g[8]);
            }
            const float hc0 = h[0];
            const float hcA = h[1] * vx + h[2] * vy + h[3] * vz;
            const float hcS = h[4] * bxx + h[5] * byy + h[6] * bxy + h[7] * bxz + h[8] * byz;
            b_phi = fmaf(Zji, hc0 * F0 + hcA * F1 + hcS * F2, b_phi);
            {
                const float cA = phi * Zji * F1, cS = phi * Zji * F2;
                bx += cA * h[1] + cS * (2.f * vx * h[4] + vy * h[6] + vz * h[7]);
                by += cA * h[2] + cS * (2.f * vy * h[5] + vx * h[6] + vz * h[8]);
                bz += cA * h[3] + cS * (vx * h[7] + vy * h[8]);
            }
            o[0][k] = phi * (Zij * gc0 + Zji * hc0);
            o[1][k] = phi * (Zij * gcA + Zji * hcA);
            o[2][k] = phi * (Zij * gcS + Zji * hcS);
        }
#pragma unroll
        for (int pl = 0; pl < 3; ++pl) {
            st4(gfu + fb + pl * F, make_float4(o[pl][0], o[pl][1], o[pl][2], o[pl][3]));
            if (gfu_cp.mode) {
#pragma unroll
                for (int k = 0; k < 4; ++k) opcopy_store(gfu_cp, fb + pl * F + k, o[pl][k]);
            }
        }
        a_phi = warp_sum(a_phi); ax = warp_sum(ax); ay = warp_sum(ay); az = warp_sum(az);
        b_phi = warp_sum(b_phi); bx = warp_sum(bx); by = warp_sum(by); bz = warp_sum(bz);
        if (lane == 0) {
            const int e = ue[u];
            edge_g[e] = make_float4(a_phi, ax, ay, az);
            edge_g[rev[e]] = make_float4(b_phi, bx, by, bz);
        }
    }
}

// dE/dr_ij of each undirected pair (i < j): one warp per pair, lane k < K.
//   dE/dd   = sum_k ge[u][k] de_k/dd + (gphi_mlp[u] + gphi(i,j) + gphi(j,i)) dphi/dd
//             + dEdd[u]  (the tabulated functions' share, table mode)
//   dE/du   = gu(i,j) - gu(j,i)                       (u_ji = -u_ij)
//   Gp[u]   = dE/dd u + (dE/du - (dE/du . u) u) / d
__global__ void k_pair_vec(const float *__restrict__ pos, const float *__restrict__ box,
                           const int32_t *__restrict__ batch, const int2 *__restrict__ uij,
                           const int32_t *__restrict__ ue, const int32_t *__restrict__ rev,
                           const int32_t *__restrict__ nu, RadialParams rp, const float *__restrict__ ge,
                           const float *__restrict__ gphi_mlp, const float4 *__restrict__ edge_g,
                           const float *__restrict__ dEdd, float *__restrict__ Gp) {
    pdl_entry();
    const int U = *nu;
    // one thread per pair (a warp keeps 32 pairs' loads in flight); the
    // pair's row of dE/de is read as float4 when K allows
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < U; u += (int64_t)gridDim.x * blockDim.x) {
        const int2 p = uij[u];
        float x, y, zz;
        pair_vec(pos, box, batch, p.x, p.y, x, y, zz);
        const float d = sqrtf(norm2_rn(x, y, zz));
        const float phi = cutoff_phi(d, rp), dphi = cutoff_dphi(d, rp);
        float s = 0.f;
        if (ge) {
            const float *g = ge + u * rp.K;
            if ((rp.K & 3) == 0) {
                for (int k = 0; k < rp.K; k += 4) {
                    const float4 gv = *reinterpret_cast<const float4 *>(g + k);
                    const float gk[4] = {gv.x, gv.y, gv.z, gv.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float e, de;
                        expnorm_k(d, k + j, rp, phi, dphi, e, de);
                        s = fmaf(gk[j], de, s);
                    }
                }
            } else {
                for (int k = 0; k < rp.K; ++k) {
                    float e, de;
                    expnorm_k(d, k, rp, phi, dphi, e, de);
                    s = fmaf(g[k], de, s);
                }
            }
        }
        {
            const int e = ue[u];
            const float4 a = edge_g[e], b = edge_g[rev[e]];
            const float gphi = (gphi_mlp ? gphi_mlp[u] : 0.f) + a.x + b.x;
            const float gd = s + gphi * dphi + (dEdd ? dEdd[u] : 0.f);
            const float inv = 1.0f / d;
            const float ux = x * inv, uy = y * inv, uz = zz * inv;
            const float gx = a.y - b.y, gy = a.z - b.z, gz = a.w - b.w;
            const float dot = gx * ux + gy * uy + gz * uz;
            Gp[3 * u] = gd * ux + (gx - dot * ux) * inv;
            Gp[3 * u + 1] = gd * uy + (gy - dot * uy) * inv;
            Gp[3 * u + 2] = gd * uz + (gz - dot * uz) * inv;
        }
    }
}

// F_i = -dE/dr_i = -sum over the active edges of row i of +-Gp[pair]
// (+ when i is the pair's first atom, r_ij = r_i - r_j), in row order.
__global__ void k_forces(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                         const int32_t *__restrict__ pair_of, const float *__restrict__ Gp, int N,
                         float *__restrict__ forces) {
    pdl_entry();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        const int u = pair_of[e];
        if (u < 0) continue;
        const float sgn = col[e] > i ? 1.0f : -1.0f;
        fx = fmaf(sgn, Gp[3LL * u], fx);
        fy = fmaf(sgn, Gp[3LL * u + 1], fy);
        fz = fmaf(sgn, Gp[3LL * u + 2], fz);
    }
    forces[3LL * i] = -fx;
    forces[3LL * i + 1] = -fy;
    forces[3LL * i + 2] = -fz;
}

// Per-element sums of the pair-embedding adjoints (split over atom ranges):
// zpart[s][0][z][c] = sum_{i in split s, z_i = z} gA_atom[i][c], and [1] for gB.
__global__ void k_group_z(const int32_t *__restrict__ z, const float *__restrict__ gA,
                          const float *__restrict__ gB, int N, int F, int max_z, int splits,
                          float *__restrict__ zpart) {
    pdl_entry();
    const int zz = blockIdx.x, s = blockIdx.y, c = threadIdx.x;
    const int chunk = (N + splits - 1) / splits;
    const int i0 = s * chunk, i1 = min(N, i0 + chunk);
    float a = 0.f, b = 0.f;
    for (int i = i0; i < i1; ++i) {
        if (z[i] == zz) {
            a += gA[(int64_t)i * F + c];
            b += gB[(int64_t)i * F + c];
        }
    }
    zpart[(((int64_t)s * 2 + 0) * max_z + zz) * F + c] = a;
    zpart[(((int64_t)s * 2 + 1) * max_z + zz) * F + c] = b;
}

// A[z] = sum over splits of the receiver sums, B[z] likewise for senders.
__global__ void k_zreduce(const float *__restrict__ zpart, int splits, int F, int max_z, float *__restrict__ AB) {
    pdl_entry();
    const int zz = blockIdx.x, c = threadIdx.x;
    for (int h = 0; h < 2; ++h) {
        float acc = 0.f;
        for (int s = 0; s < splits; ++s) acc += zpart[(((int64_t)s * 2 + h) * max_z + zz) * F + c];
        AB[((int64_t)h * max_z + zz) * F + c] = acc;
    }
}

// Gradients of the atom embedding and the pair embedding Linear from the
// per-element sums A[z] (receiver) and B[z] (sender), Z_ij = W_e[emb_zi; emb_zj] + b_e.
// Blocks 0..F-1 give rows of dW_e (and db_e), blocks F..F+max_z-1 rows of demb.
__global__ void k_emb_tables_grad2(const float *__restrict__ AB, int F, int max_z, const float *__restrict__ emb,
                                   const float *__restrict__ We, float *__restrict__ g_emb,
                                   float *__restrict__ g_We, float *__restrict__ g_be) {
    pdl_entry();
    const int r = blockIdx.x, c = threadIdx.x;
    const float *A = AB, *B = AB + (int64_t)max_z * F;
    if (r < F) {
        // g_We[r][c] = sum_z A[z][r] emb[z][c];  g_We[r][F + c] = sum_z B[z][r] emb[z][c]
        float a = 0.f, b = 0.f;
        for (int zz = 0; zz < max_z; ++zz) {
            const float e = emb[(int64_t)zz * F + c];
            a = fmaf(A[(int64_t)zz * F + r], e, a);
            b = fmaf(B[(int64_t)zz * F + r], e, b);
        }
        g_We[(int64_t)r * 2 * F + c] = a;
        g_We[(int64_t)r * 2 * F + F + c] = b;
        if (r == 0) {
            float bb = 0.f;
            for (int zz = 0; zz < max_z; ++zz) bb += A[(int64_t)zz * F + c];
            g_be[c] = bb;
        }
    } else {
        // g_emb[z][c] = sum_r A[z][r] We[r][c] + B[z][r] We[r][F + c]
        const int zz = r - F;
        float a = 0.f;
        for (int q = 0; q < F; ++q)
            a += A[(int64_t)zz * F + q] * We[(int64_t)q * 2 * F + c] + B[(int64_t)zz * F + q] * We[(int64_t)q * 2 * F + F + c];
        g_emb[(int64_t)zz * F + c] = a;
    }
}

// dE/dE_i (seed of the system) and its products for the head gradients
__global__ void k_seed_atoms(const float *__restrict__ seed, const int32_t *__restrict__ batch, int N,
                             float *__restrict__ gEi) {
    pdl_entry();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) gEi[i] = seed ? seed[batch ? batch[i] : 0] : 1.0f;
}

// Plane-major copy of each layer's last radial-MLP layer: row p*F + c of the
// copy is row c*3 + p of the blob (weight [3F][2F], then bias [3F]), so the
// per-pair filters g_ij and their adjoints are three contiguous F-channel
// planes I, A, S and the message kernels read and write them coalesced.
struct FilterRows {
    const float *w[8], *b[8];
};
__global__ void k_filter_rows(const __grid_constant__ FilterRows R, int F, float *__restrict__ out) {
    pdl_entry();
    const int l = blockIdx.y;
    const int64_t nw = 6LL * F * F, per = nw + 3 * F;
    const int cols = 2 * F;
    float *o = out + l * per;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < per; t += (int64_t)gridDim.x * blockDim.x) {
        if (t < nw) {
            const int r = (int)(t / cols), k = (int)(t % cols);
            o[t] = R.w[l][(int64_t)((r % F) * 3 + r / F) * cols + k];
        } else {
            const int r = (int)(t - nw);
            o[t] = R.b[l][(r % F) * 3 + r / F];
        }
    }
}

// Weight operands of the tensor-core modes: job j reads a [rows][cols] float
// matrix (transposed when tr[j], for backward operands) and writes a bf16
// copy (mode[j] = 1) or its TF32 split hi + lo (mode[j] = 2, the 3xTF32
// GEMMs).
constexpr int kMaxCvtJobs = 128;
struct CvtJobs {
    const float *src[kMaxCvtJobs];
    void *hi[kMaxCvtJobs];
    void *lo[kMaxCvtJobs];
    int rows[kMaxCvtJobs], cols[kMaxCvtJobs], tr[kMaxCvtJobs], mode[kMaxCvtJobs];
    int n;
};
struct WOp {  // a weight operand: bf16 matrix, or fp32 high part + residual
    const void *b;
    const void *blo;
};
__global__ void k_cvt_weights(const __grid_constant__ CvtJobs J) {
    pdl_entry();
    const int j = blockIdx.y;
    if (j >= J.n) return;
    const int R = J.rows[j], C = J.cols[j];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < R * C; t += gridDim.x * blockDim.x) {
        const int r = t / C, c = t % C;
        const float v = J.src[j][t];
        const int64_t o = J.tr[j] ? (int64_t)c * R + r : (int64_t)t;
        if (J.mode[j] == 1) {
            static_cast<__nv_bfloat16 *>(J.hi[j])[o] = __float2bfloat16_rn(v);
        } else {
            float hi, lo;
            tf32_split(v, hi, lo);
            static_cast<float *>(J.hi[j])[o] = hi;
            static_cast<float *>(J.lo[j])[o] = lo;
        }
    }
}

// Per-context kernel set-up (nothing needs opting in at present).
int tnet_kernel_setup(tnet_ctx *c) {
    (void)c;
    return TNET_OK;
}

// Tensor-core GEMM with the column tile chosen from N.
template <class Epi>
int tc_any(const tc::TcShape &P, const __nv_bfloat16 *A, int64_t a_rows, int64_t lda, const __nv_bfloat16 *B,
           int64_t b_rows, int64_t ldb, const Epi &epi, int32_t *status, cudaStream_t st, int sms, int bn = 0) {
    if (bn == 128 && P.N % 128 == 0) return tc::tc_gemm<128>(P, A, a_rows, lda, B, b_rows, ldb, epi, status, st, sms);
    if (bn == 192 && P.N % 192 == 0) return tc::tc_gemm<192>(P, A, a_rows, lda, B, b_rows, ldb, epi, status, st, sms);
    if (bn == 256 && P.N % 256 == 0) return tc::tc_gemm<256>(P, A, a_rows, lda, B, b_rows, ldb, epi, status, st, sms);
    if (P.N <= 32) return tc::tc_gemm<32>(P, A, a_rows, lda, B, b_rows, ldb, epi, status, st, sms);
    if (P.N <= 64) return tc::tc_gemm<64>(P, A, a_rows, lda, B, b_rows, ldb, epi, status, st, sms);
    if (P.N <= 128) return tc::tc_gemm<128>(P, A, a_rows, lda, B, b_rows, ldb, epi, status, st, sms);
    if (P.N % 256 == 0) return tc::tc_gemm<256>(P, A, a_rows, lda, B, b_rows, ldb, epi, status, st, sms);
    if (P.N % 192 == 0) return tc::tc_gemm<192>(P, A, a_rows, lda, B, b_rows, ldb, epi, status, st, sms);
    if (P.N % 128 == 0) return tc::tc_gemm<128>(P, A, a_rows, lda, B, b_rows, ldb, epi, status, st, sms);
    return TNET_ERR_ARG;
}

// Launch the thread-per-channel row kernels with 4 consecutive rows per block
// when rb >= 4 and the block fits (at most 1024 threads for the messages, 512
// for their adjoint, whose per-row staging is 37 KB at F = 128), else one.
// blocks1 is the grid the one-row-per-block launch would use.
template <int F, bool TAB, class... Args>
static void launch_message(int rb, int blocks1, cudaStream_t st, Args... args) {
    if constexpr (F * 4 <= 1024) {
        if (rb >= 4) {
            launch(k_message<F, TAB, 4>, (blocks1 + 3) / 4, F * 4, 0, st, args...);
            return;
        }
    }
    launch(k_message<F, TAB, 1>, blocks1, F, 0, st, args...);
}
template <int F, bool TAB, class... Args>
static void launch_message_bwd(int rb, int blocks1, cudaStream_t st, Args... args) {
    if constexpr (F * 4 <= 512) {
        if (rb >= 4) {
            launch(k_message_bwd<F, TAB, 4>, (blocks1 + 3) / 4, F * 4, 0, st, args...);
            return;
        }
    }
    launch(k_message_bwd<F, TAB, 1>, blocks1, F, 0, st, args...);
}

// ============================================== host-side launch sequence ===
static inline int grid_for(int64_t n, int threads, int num_sms) {
    int64_t g = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms * 16;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

#define TRY(...)                    \
    do {                            \
        int rc_ = (__VA_ARGS__);    \
        if (rc_) return rc_;        \
    } while (0)

// Row offsets clamped to [0, cap] (cap = the context's pair capacity, which
// sizes every per-edge buffer): a caller's CSR can then never send a kernel
// outside those buffers.  Offsets outside the range or decreasing are
// reported as ARG (or CAPACITY when they pass the capacity).
__global__ void k_rows_in_range(const int32_t *__restrict__ row_ptr, int N, int64_t cap,
                                int32_t *__restrict__ safe, int32_t *status) {
    pdl_entry();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t <= N; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = row_ptr[t];
        int32_t w = v < 0 ? 0 : v;
        if (w > cap) {
            w = (int32_t)cap;
            set_status(status, TNET_ERR_CAPACITY);
        }
        if (v < 0 || (t == 0 && v != 0) || (t > 0 && row_ptr[t - 1] > v)) set_status(status, TNET_ERR_ARG);
        safe[t] = w;
    }
}

// Radial-function tables (radial_table = n > 0): the projections f (table 0)
// and each layer's filter g (table 1 + l) as [n-1][4][3F] Hermite
// coefficients on the grid d_k = k h, h = rc/(n - 1).  f, g are functions of
// the pair distance alone (the expnorm basis, the cosine cutoff and the radial
// MLP of TensorNet Sec. 2.1.1); the chain runs in FP64 on the values and
// their d-derivatives.
int radial_tables_impl(tnet_ctx *ctx, const float *wblob, cudaStream_t st) {
    const tnet_model_desc &d = ctx->d;
    const Layout &Lw = ctx->lay;
    const int F = d.F, K = d.K, NL = d.L, nt = d.radial_table;
    const int sms = ctx->num_sms;
    if (nt <= 0) return TNET_ERR_ARG;
    Weights W;
    weight_offsets(&d, wblob, &W);
    auto f32 = [&](size_t off) { return wsp<float>(ctx, off); };
    const double rc = d.cutoff_upper, rl = d.cutoff_lower;
    RadialParams64 rp{rc, rl, 5.0 / (rc - rl), pow((2.0 / K) * (1.0 - exp(-(rc - rl))), -2.0), exp(-(rc - rl)),
                      (1.0 - exp(-(rc - rl))) / (K - 1), K};
    const double h = rc / (nt - 1);
    const int64_t per_fn = (int64_t)(nt - 1) * 4 * 3 * F;
    auto coef = [&](int j) { return reinterpret_cast<float4 *>(f32(Lw.tab) + j * per_fn); };
    const int64_t w3_per = 6LL * F * F + 3 * F;
    auto w3p = [&](int l) { return f32(Lw.w3p) + l * w3_per; };
    auto b3p = [&](int l) { return f32(Lw.w3p) + l * w3_per + 6LL * F * F; };
    if (NL > 0) {
        FilterRows FR{};
        for (int l = 0; l < NL; ++l) { FR.w[l] = W.layer[l].mlp3_w; FR.b[l] = W.layer[l].mlp3_b; }
        launch(k_filter_rows, dim3(48, NL), 256, 0, st, FR, F, f32(Lw.w3p));
        count_launch();
        TNET_LAUNCH_CHECK();
    }
    double *e_t = wsp<double>(ctx, Lw.tab_tmp), *de_t = e_t + (int64_t)nt * K, *phi_t = de_t + (int64_t)nt * K,
           *dphi_t = phi_t + nt, *h1_t = dphi_t + nt, *t1_t = h1_t + (int64_t)nt * F, *h2_t = t1_t + (int64_t)nt * F,
           *t2_t = h2_t + (int64_t)nt * 2 * F, *v_t = t2_t + (int64_t)nt * 2 * F, *dv_t = v_t + (int64_t)nt * 3 * F;
    launch(k_tab_rbf, grid_for((int64_t)nt * K, 256, sms), 256, 0, st, nt, h, rp, e_t, de_t, phi_t, dphi_t);
    count_launch();
    TNET_LAUNCH_CHECK();
    auto layer = [&](int Nout, int Kin, const double *x, const double *tx, const float *w, const float *b, int mode,
                     double *y, double *ty) {
        launch(k_tab_layer, dim3((Nout + 63) / 64, (nt + 63) / 64), 256, 0, st, nt, Nout, Kin, x, tx, w, b, mode,
               phi_t, dphi_t, y, ty);
        count_launch();
    };
    auto finish = [&](int j) {
        launch(k_tab_coef, grid_for((int64_t)(nt - 1) * 3 * F, 256, sms), 256, 0, st, nt, 3 * F, h, v_t, dv_t,
               coef(j));
        count_launch();
    };
    layer(3 * F, K, e_t, de_t, W.dproj_w, W.dproj_b, 1, v_t, dv_t);
    finish(0);
    for (int l = 0; l < NL; ++l) {
        const LayerW &Lr = W.layer[l];
        layer(F, K, e_t, de_t, Lr.mlp1_w, Lr.mlp1_b, 0, h1_t, t1_t);
        layer(2 * F, F, h1_t, t1_t, Lr.mlp2_w, Lr.mlp2_b, 0, h2_t, t2_t);
        layer(3 * F, 2 * F, h2_t, t2_t, w3p(l), b3p(l), 2, v_t, dv_t);
        finish(1 + l);
    }
    TNET_LAUNCH_CHECK();
    ctx->tab_ready = 1;
    return TNET_OK;
}

int energy_forces_impl(tnet_ctx *ctx, const float *wblob, int N, int S, const int32_t *z,
                       const float *pos, const int32_t *batch, const float *box,
                       const int32_t *row_ptr_in, const int32_t *col, const float *seed,
                       double *energy, float *forces, float *grad_w, int32_t *status,
                       cudaStream_t st) {
    const tnet_model_desc &d = ctx->d;
    const Layout &Lw = ctx->lay;
    const int F = d.F, K = d.K, NL = d.L, H = F / 2;
    // table mode: the radial functions are tabulated, which has no weight adjoint
    const int nt = d.radial_table;
    const bool tab = nt > 0;
    if (tab && grad_w) return TNET_ERR_UNSUPPORTED;
    const float th = tab ? ctx->rp.rc / (float)(nt - 1) : 0.f;
    const int sms = ctx->num_sms;
    const RadialParams rp = ctx->rp;
    const int gctas = sms * ctx->tune[T_GEMM_CTAS];
    const int bn3 = ctx->tune[T_TC_BN_3F], bn2 = ctx->tune[T_TC_BN_2F];
    const int pair_grid = sms * ctx->tune[T_PAIR_BLOCKS];
    Weights W, G;
    weight_offsets(&d, wblob, &W);
    weight_offsets(&d, grad_w, &G);
    auto gw = [](const float *p) { return const_cast<float *>(p); };
    auto f32 = [&](size_t off) { return wsp<float>(ctx, off); };
    auto i32 = [&](size_t off) { return wsp<int32_t>(ctx, off); };
    const int64_t n9 = Lw.node9;
    const int maxU = (int)Lw.maxU;
    float *wpart = f32(Lw.wpart);
    const int64_t wcap = Lw.wpart_floats;
    int32_t *sys_start = i32(Lw.sys_start), *sys_end = i32(Lw.sys_end);
    int32_t *rev = i32(Lw.rev), *pair_of = i32(Lw.pair_of), *ucnt = i32(Lw.ucnt);
    // every kernel below reads the clamped copy of the row offsets
    int32_t *row_ptr = i32(Lw.rp_safe);
    launch(k_rows_in_range, (N + 256) / 256 < 1024 ? (N + 256) / 256 : 1024, 256, 0, st, row_ptr_in, N,
           ctx->max_pairs, row_ptr, status);
    count_launch();
    TNET_LAUNCH_CHECK();
    int32_t *nu = i32(Lw.nu), *ue = i32(Lw.ue);
    int2 *uij = wsp<int2>(ctx, Lw.uedge);
    float *Ta = f32(Lw.Ta), *Tb = f32(Lw.Tb);
    const int warps_grid = (int)(((int64_t)N * 32 + 255) / 256);
    // row-sum shapes for weight gradients
    auto rows1 = [&](int M_, int N_, int64_t R, const float *A, int64_t lda, const float *B, int64_t ldb,
                     const int32_t *rows_dev) {
        WgradShape P{};
        P.M = M_; P.N = N_; P.rows[0] = R; P.row0[0] = 0; P.rows_dev = rows_dev; P.rows_mul = 1;
        P.A = A; P.lda = lda; P.B = B; P.ldb = ldb; P.nclass = 1;
        return P;
    };
    auto rows3 = [&](const float *A, const float *B) {  // the I, A, S coordinate planes
        WgradShape P{};
        P.M = F; P.N = F;
        P.rows[0] = N; P.rows[1] = 3LL * N; P.rows[2] = 5LL * N;
        P.row0[0] = 0; P.row0[1] = N; P.row0[2] = 4LL * N;
        P.rows_dev = nullptr; P.rows_mul = 1;
        P.A = A; P.lda = F; P.B = B; P.ldb = F; P.nclass = 3;
        return P;
    };

    // ---- tensor-core modes: operand copies and weight copies
    //   precision 1 (BF16): bf16 operands, one MMA per k-step
    //   precision 2 (3xTF32): fp32 operands plus their TF32 residuals
    const int prec = d.precision;
    const bool tcm = prec != 0;
    const bool wg = grad_w != nullptr;
    // FP32 activations h1, h2 are read by the FP32 GEMMs and by the weight
    // gradients (the 3xTF32 GEMMs form them from a1, a2 when no weight
    // gradient is asked for); the BF16 GEMMs read only their bf16 copies
    const bool keep_h = prec != 1 || wg;
    // bf16 operand copies (BF16 mode only: the 3xTF32 GEMMs read the fp32
    // activations and form their residuals on chip)
    auto cp = [&](size_t off) { return prec == 1 ? OpCopy{(void *)(ctx->ws + off), 1} : OpCopy{nullptr, 0}; };
    // (the num_rbf-wide operands e(d) and dE/df stay FP32, so they get no copy)
    const OpCopy none{nullptr, 0};
    const OpCopy nbf = cp(Lw.nbf), eu_cp = none, ga3_cp = cp(Lw.ga3_bf), ga2_cp = cp(Lw.ga2_bf), ga1_cp = none,
                 gfu_cp = none;
    // per-layer radial-MLP activations (and their operand copies)
    const int64_t esz_cp = 2;
    // slab of layer l (one shared slab when the reverse pass recomputes them)
    const bool keep_act = !d.recompute_edges;
    auto slab = [&](int l) { return keep_act ? (int64_t)l : 0; };
    auto h1_cp = [&](int l) { return cp(Lw.h1_bf + (size_t)(slab(l) * maxU * F * esz_cp)); };
    auto h2_cp = [&](int l) { return cp(Lw.h2_bf + (size_t)(slab(l) * maxU * 2 * F * esz_cp)); };
    struct LayerB {
        WOp mlp2, mlp3, mlp2T, mlp3T, mix1, mix1T, mix2, mix2T, mlp1, mlp1T;
    } lb[8] = {};
    WOp emix{}, emixT{};
    // 3xTF32 weight operands of the num_rbf-wide radial layers, in both
    // tensor-core modes (rounding the narrow expnorm basis to bf16 costs more
    // force accuracy than any other operand), and of the per-atom embedding
    // and output MLPs in BF16 mode.  In the FP32-accurate mode those per-atom
    // MLPs stay on FP32 FMA: they are cheap, and the energy is the quantity
    // most sensitive to them (3xTF32 there costs an order of magnitude of
    // energy accuracy).
    const bool atom_x3 = prec == 1;
    struct X3W {
        WOp dproj, dprojT, emb_mlp1, emb_mlp1T, emb_mlp2, emb_mlp2T, out, outT, head1, head1T;
    } wx{};

    // ---- graph prep
    ProfSeq pf(ctx, st);
    pf.mark(P_PREP);
    const int64_t w3_per = 6LL * F * F + 3 * F;
    auto w3p = [&](int l) { return f32(Lw.w3p) + l * w3_per; };  // plane-major mlp3 weight
    auto b3p = [&](int l) { return f32(Lw.w3p) + l * w3_per + 6LL * F * F; };
    if (NL > 0 && !tab) {
        FilterRows FR{};
        for (int l = 0; l < NL; ++l) { FR.w[l] = W.layer[l].mlp3_w; FR.b[l] = W.layer[l].mlp3_b; }
        launch(k_filter_rows, dim3(48, NL), 256, 0, st, FR, F, f32(Lw.w3p));
        count_launch();
        TNET_LAUNCH_CHECK();
    }
    if (tcm) {
        CvtJobs J;
        J.n = 0;
        char *wb = ctx->ws + Lw.wbf;
        int64_t woff = 0;  // bytes
        auto alloc = [&](int64_t elems, int esz) {
            void *p = wb + woff;
            woff += (elems * esz + 255) & ~(int64_t)255;
            return p;
        };
        // forward operands keep the (out, in) = K-major layout; backward
        // operands are transposed
        auto job_m = [&](const float *src, int rows, int cols, int tr, int mode) {
            WOp w{};
            const int esz = mode == 1 ? 2 : 4;
            void *hi = alloc((int64_t)rows * cols, esz);
            void *lo = mode == 2 ? alloc((int64_t)rows * cols, esz) : nullptr;
            J.src[J.n] = src; J.hi[J.n] = hi; J.lo[J.n] = lo;
            J.rows[J.n] = rows; J.cols[J.n] = cols; J.tr[J.n] = tr; J.mode[J.n] = mode;
            ++J.n;
            w.b = hi;
            w.blo = lo;
            return w;
        };
        auto job = [&](const float *src, int rows, int cols, int tr) { return job_m(src, rows, cols, tr, prec); };
        auto job3 = [&](const float *src, int rows, int cols, int tr) { return job_m(src, rows, cols, tr, 2); };
        // [3][F][F] -> per-class transposes; the three classes' high parts (and
        // residuals) must stay stacked contiguously [3F][F] for the GEMM
        auto job_classes_T = [&](const float *src) {
            const int64_t ff = (int64_t)F * F;
            const int esz = prec == 1 ? 2 : 4;
            char *hi = (char *)alloc(3 * ff, esz), *lo = prec == 2 ? (char *)alloc(3 * ff, esz) : nullptr;
            for (int q = 0; q < 3; ++q) {
                J.src[J.n] = src + q * ff;
                J.hi[J.n] = hi + q * ff * esz;
                J.lo[J.n] = lo ? lo + q * ff * esz : nullptr;
                J.rows[J.n] = F; J.cols[J.n] = F; J.tr[J.n] = 1; J.mode[J.n] = prec;
                ++J.n;
            }
            return WOp{hi, lo};
        };
        emix = job(W.emb_mix_w, 3 * F, F, 0);
        emixT = job_classes_T(W.emb_mix_w);
        for (int l = 0; l < NL; ++l) {
            const LayerW &Lr = W.layer[l];
            lb[l].mix1 = job(Lr.mix1_w, 3 * F, F, 0);
            lb[l].mix1T = job_classes_T(Lr.mix1_w);
            lb[l].mix2 = job(Lr.mix2_w, 3 * F, F, 0);
            lb[l].mix2T = job_classes_T(Lr.mix2_w);
            if (tab) continue;  // no per-pair radial MLP
            lb[l].mlp2 = job(Lr.mlp2_w, 2 * F, F, 0);
            lb[l].mlp3 = job(w3p(l), 3 * F, 2 * F, 0);
            lb[l].mlp2T = job(Lr.mlp2_w, 2 * F, F, 1);
            lb[l].mlp3T = job(w3p(l), 3 * F, 2 * F, 1);
            lb[l].mlp1 = job3(Lr.mlp1_w, F, K, 0);
            lb[l].mlp1T = job3(Lr.mlp1_w, F, K, 1);
        }
        if (!tab) {
            wx.dproj = job3(W.dproj_w, 3 * F, K, 0);
            wx.dprojT = job3(W.dproj_w, 3 * F, K, 1);
        }
        if (atom_x3) {
            wx.emb_mlp1 = job3(W.emb_mlp1_w, 2 * F, F, 0);
            wx.emb_mlp1T = job3(W.emb_mlp1_w, 2 * F, F, 1);
            wx.emb_mlp2 = job3(W.emb_mlp2_w, 3 * F, 2 * F, 0);
            wx.emb_mlp2T = job3(W.emb_mlp2_w, 3 * F, 2 * F, 1);
            wx.out = job3(W.out_w, F, 3 * F, 0);
            wx.outT = job3(W.out_w, F, 3 * F, 1);
            wx.head1 = job3(W.head1_w, H, F, 0);
            wx.head1T = job3(W.head1_w, H, F, 1);
        }
        if (woff > Lw.wbf_bytes || J.n > kMaxCvtJobs) return TNET_ERR_WORKSPACE;
        launch(k_cvt_weights, dim3(64, J.n), 256, 0, st, J);
        count_launch();
        TNET_LAUNCH_CHECK();
    }
    // 3xTF32 tensor-core GEMM: fp32 A (split in the kernel) against weight
    // operand w (its TF32 split)
    auto tcx3 = [&](const tc::TcShape &P0, const float *A32, int64_t a_rows, int64_t lda, const WOp &w,
                    int64_t b_rows, int64_t ldb, const auto &epi, int bn = 0) -> int {
        const tc::TcOperands o{A32, w.b, w.blo, a_rows, lda, b_rows, ldb};
        tc::TcShape P = P0;
        P.cl = ctx->tune[T_TC_CLUSTER];
        if (P.N <= 32) return tc::tc_gemm_ops<32, true>(P, o, epi, status, st, sms);
        if (P.N <= 64) return tc::tc_gemm_ops<64, true>(P, o, epi, status, st, sms);
        // num_rbf-deep GEMMs (radial layer 1, the projections) are bound by
        // their epilogue, not their MMAs: they keep sixteen epilogue warps
        if (P.K <= 32) {
            if (P.N % 192 == 0 && bn != 128) return tc::tc_gemm_ops<192, true, true>(P, o, epi, status, st, sms);
            return tc::tc_gemm_ops<128, true, true>(P, o, epi, status, st, sms);
        }
        // 2F-wide outputs: one 256-wide tile when the knob asks for it (fewer
        // tile loads per MMA: 40 KB of TMA per 880 MMA cycles against 24 KB per
        // 440 at 128)
        if (P.N % 256 == 0 && bn == 256) return tc::tc_gemm_ops<256, true>(P, o, epi, status, st, sms);
        if (P.N % 192 == 0 && bn != 128) return tc::tc_gemm_ops<192, true>(P, o, epi, status, st, sms);
        return tc::tc_gemm_ops<128, true>(P, o, epi, status, st, sms);
    };
    // tensor-core GEMM of the mode: BF16 (A's bf16 copy) or 3xTF32 (A itself)
    auto tcg = [&](const tc::TcShape &P, const float *A32, const OpCopy &Acp, int64_t a_rows, int64_t lda,
                   const WOp &w, int64_t b_rows, int64_t ldb, const auto &epi, int bn = 0) -> int {
        if (prec == 1) {
            tc::TcShape Q = P;
            Q.cl = ctx->tune[T_TC_CLUSTER];
            return tc_any(Q, (const __nv_bfloat16 *)Acp.p, a_rows, lda, (const __nv_bfloat16 *)w.b, b_rows, ldb,
                          epi, status, st, sms, bn);
        }
        return tcx3(P, A32, a_rows, lda, w, b_rows, ldb, epi, bn);
    };
    TNET_CUDA_TRY(cudaMemsetAsync(sys_start, 0, sizeof(int32_t) * S, st));
    TNET_CUDA_TRY(cudaMemsetAsync(sys_end, 0, sizeof(int32_t) * S, st));
    TRY(sys_bounds(batch, N, S, sys_start, sys_end, status, st));
    launch(k_rev, warps_grid, 256, 0, st, row_ptr, col, N, rev, status);
    count_launch();
    launch(k_upper_count, warps_grid, 256, 0, st, pos, box, batch, row_ptr, col, N, rp.rc, ucnt);
    count_launch();
    TNET_LAUNCH_CHECK();
    TRY(scan_exclusive_i32(ucnt, ucnt, N, i32(Lw.scan_tmp), nu, nullptr, st));
    launch(k_upper_assign, warps_grid, 256, 0, st, pos, box, batch, row_ptr, col, N, rp.rc, ucnt, pair_of, uij, ue);
    count_launch();
    launch(k_lower_assign, warps_grid, 256, 0, st, row_ptr, col, rev, N, pair_of);
    count_launch();
    TNET_LAUNCH_CHECK();
    float *eu = f32(Lw.eu), *phiu = f32(Lw.phiu), *fu = f32(Lw.fu);
    float4 *geo = wsp<float4>(ctx, Lw.geo);
    // table mode: function 0 is the projections f, function 1 + l layer l's
    // filter g, each [n-1][3F] float4 Hermite coefficients
    float *dist = f32(Lw.dist);
    auto tabfn = [&](int j) {
        if (!tab) return TabFn{nullptr, nullptr, 0, 0.f};
        return TabFn{reinterpret_cast<const float4 *>(f32(Lw.tab) + (int64_t)j * (nt - 1) * 4 * 3 * F), dist, nt,
                     1.0f / th};
    };
    const TabFn tf0 = tabfn(0);
    if (tab) {
        if (!ctx->tab_ready) return TNET_ERR_ARG;  // tnet_radial_tables not called
        launch(k_pair_geo, grid_for(maxU, 256, sms), 256, 0, st, pos, box, batch, uij, nu, rp, phiu, geo, dist);
        count_launch();
    } else {
        launch(k_edge_rbf, pair_grid, 256, 0, st, pos, box, batch, uij, nu, maxU, rp, eu, phiu, geo, eu_cp);
        count_launch();
    }
    launch(k_elem_tables, d.max_z, 256, sizeof(float) * F, st, W.emb, W.emb2_w, W.emb2_b, F, Ta, Tb);
    count_launch();
    TNET_LAUNCH_CHECK();
    if (!tab) {   // radial projections f^p = W^p e(d) + b^p, once per undirected pair
        // FP32 in both modes: K = num_rbf is small, and rounding the narrow
        // expnorm basis values to bf16 costs more force accuracy than any
        // other operand
        const EpiBiasAct ep{W.dproj_b, nullptr, 0, fu, 3 * F, 0, nullptr};
        if (tcm) {
            tc::TcShape tp = tc::tshape(maxU, 3 * F, K);
            tp.rows_dev = nu;
            TRY(tcx3(tp, eu, maxU, K, wx.dproj, 3 * F, K, ep, bn3));
        } else {
            GemmShape pp = gshape(maxU, 3 * F, K, eu, K, W.dproj_w, K);
            pp.rows_dev = nu;
            TRY(sgemm<false, true>(pp, ep, gctas, st));
        }
    }

    // ---- embedding
    pf.mark(P_EMB_EDGE);
    float *Xraw = f32(Lw.Xraw), *Uemb = f32(Lw.Uemb), *n0 = f32(Lw.n0), *as1 = f32(Lw.as1),
          *hs1 = f32(Lw.hs1), *as2 = f32(Lw.as2), *s = f32(Lw.s), *q0 = f32(Lw.q0);
    float2 *ln0 = wsp<float2>(ctx, Lw.ln0);
    const int atom_blocks = N < sms * ctx->tune[T_ROW_BLOCKS] ? N : sms * ctx->tune[T_ROW_BLOCKS];
    // message kernels (and the pair-parallel embedding adjoint): knob 0 =
    // one warp per row (pair) with four channels per lane (exact mode,
    // F = 128, 32-bit offsets; the adjoint at two blocks per SM), 3 = the
    // same with the adjoint at three blocks per SM, 1 or 4 = that many
    // consecutive rows per block of F threads (one thread per channel)
    const int rows_pb = ctx->tune[T_MSG_KERNEL] == 4 ? 4 : 1;
    const bool warp_rows = (ctx->tune[T_MSG_KERNEL] == 0 || ctx->tune[T_MSG_KERNEL] == 3) && !tab && F == 128 &&
                           9LL * N * F < (1LL << 31) && (int64_t)maxU * 3 * F < (1LL << 31);
    const int v4_blocks = (int)((N + kV4Warps - 1) / kV4Warps < atom_blocks ? (N + kV4Warps - 1) / kV4Warps
                                                                             : atom_blocks);
#define EMB_FWD(FF)                                                                                           \
    if (tab)                                                                                                  \
        launch(k_emb_edges<FF, true>, atom_blocks, FF, 0, st, geo, z, row_ptr, col, pair_of, N, d.max_z, fu, tf0, Ta, \
                                                          Tb, Xraw, status, nbf);                                   \
    else                                                                                                      \
        launch(k_emb_edges<FF, false>, atom_blocks, FF, 0, st, geo, z, row_ptr, col, pair_of, N, d.max_z, fu, tf0, Ta, \
                                                           Tb, Xraw, status, nbf)
    TNET_F_SWITCH(F, EMB_FWD);
#undef EMB_FWD
    count_launch();
    launch(k_norm_ln, N, F, 0, st, Xraw, N, F, W.emb_ln_g, W.emb_ln_b, n0, ln0, q0);
    count_launch();
    TNET_LAUNCH_CHECK();
    pf.mark(P_EMB_NODE);
    {
        const EpiBiasAct em1{W.emb_mlp1_b, as1, 2 * F, hs1, 2 * F, 1, nullptr};
        const EpiBiasAct em2{W.emb_mlp2_b, as2, 3 * F, s, 3 * F, 1, nullptr};
        if (atom_x3) {
            TRY(tcx3(tc::tshape(N, 2 * F, F), n0, N, F, wx.emb_mlp1, 2 * F, F, em1, bn2));
            TRY(tcx3(tc::tshape(N, 3 * F, 2 * F), hs1, N, 2 * F, wx.emb_mlp2, 3 * F, 2 * F, em2, bn3));
        } else {
            TRY(sgemm<false, true>(gshape(N, 2 * F, F, n0, F, W.emb_mlp1_w, F), em1, gctas, st));
            TRY(sgemm<false, true>(gshape(N, 3 * F, 2 * F, hs1, 2 * F, W.emb_mlp2_w, 2 * F), em2, gctas, st));
        }
    }
    if (tcm) TRY(tcg(tc::tshape_classes(N, F), Xraw, nbf, 9LL * N, F, emix, 3 * F, F, EpiStore{Uemb, F, 0}));
    else TRY(sgemm<false, true>(gshape_classes(N, F, Xraw, W.emb_mix_w), EpiStore{Uemb, F, 0}, gctas, st));
    float *X = f32(Lw.Xin);  // layer 0 input
    launch(k_emb_scale, grid_for((int64_t)N * F, 256, sms), 256, 0, st, Uemb, s, N, F, X);
    count_launch();
    TNET_LAUNCH_CHECK();

    // ---- interaction layers
    // layer l's radial-MLP activations: [maxU][width] slabs
    auto act = [&](size_t off, int width, int l) { return f32(off) + slab(l) * maxU * width; };
    // The radial MLP of layer l over the undirected pairs.  Its last layer
    // stores only the pre-activation a3: the message kernels form the filter
    // g = phi SiLU(a3) themselves.  fwd_only (the forward pass when the reverse
    // pass recomputes the activations): a1 and a2 are not stored, since only
    // the reverse pass reads them.
    auto edge_mlp = [&](int l, bool fwd_only) -> int {
        const LayerW &Lr = W.layer[l];
        float *a1 = act(Lw.a1, F, l), *h1 = act(Lw.h1, F, l), *a2 = act(Lw.a2, 2 * F, l),
              *h2 = act(Lw.h2, 2 * F, l), *a3 = act(Lw.a3, 3 * F, l);
        if (tab) return TNET_OK;  // the message kernels evaluate g, dg/dd from the table
        const EpiBiasAct e3{b3p(l), a3, 3 * F, nullptr, 3 * F, 0, nullptr};
        if (tcm && prec == 2 && !wg) {
            // 3xTF32 without weight gradients: layers 1 and 2 store their
            // pre-activations alone; the next GEMM's converter warps form
            // h = silu_f(a) from them (bitwise the value the epilogue would
            // store), and the reverse pass reads only a1, a2
            const EpiBiasAct s1{Lr.mlp1_b, a1, F, nullptr, F, 1, nullptr};
            const EpiBiasAct s2{Lr.mlp2_b, a2, 2 * F, nullptr, 2 * F, 1, nullptr};
            tc::TcShape t1 = tc::tshape(maxU, F, K), t2 = tc::tshape(maxU, 2 * F, F), t3 = tc::tshape(maxU, 3 * F, 2 * F);
            t1.rows_dev = t2.rows_dev = t3.rows_dev = nu;
            t2.a_silu = t3.a_silu = 1;
            pf.mark(P_MLP1);
            TRY(tcx3(t1, eu, maxU, K, lb[l].mlp1, F, K, s1));
            pf.mark(P_MLP2);
            TRY(tcx3(t2, a1, maxU, F, lb[l].mlp2, 2 * F, F, s2, bn2));
            pf.mark(P_MLP3);
            TRY(tcx3(t3, a2, maxU, 2 * F, lb[l].mlp3, 3 * F, 2 * F, e3, bn3));
            return TNET_OK;
        }
        const EpiBiasAct e1{Lr.mlp1_b, fwd_only ? nullptr : a1, F, keep_h ? h1 : nullptr, F, 1, nullptr, h1_cp(l), F};
        const EpiBiasAct e2{Lr.mlp2_b, fwd_only ? nullptr : a2, 2 * F, keep_h ? h2 : nullptr, 2 * F, 1, nullptr,
                            h2_cp(l), 2 * F};
        if (tcm) {
            tc::TcShape t2 = tc::tshape(maxU, 2 * F, F), t3 = tc::tshape(maxU, 3 * F, 2 * F);
            t2.rows_dev = t3.rows_dev = nu;
            pf.mark(P_MLP1);  // K = num_rbf: 3xTF32 in both modes (see the projections above)
            tc::TcShape t1 = tc::tshape(maxU, F, K);
            t1.rows_dev = nu;
            TRY(tcx3(t1, eu, maxU, K, lb[l].mlp1, F, K, e1));
            pf.mark(P_MLP2);
            TRY(tcg(t2, h1, h1_cp(l), maxU, F, lb[l].mlp2, 2 * F, F, e2, bn2));
            pf.mark(P_MLP3);
            TRY(tcg(t3, h2, h2_cp(l), maxU, 2 * F, lb[l].mlp3, 3 * F, 2 * F, e3, bn3));
            return TNET_OK;
        }
        pf.mark(P_MLP1);
        GemmShape p1 = gshape(maxU, F, K, eu, K, Lr.mlp1_w, K);
        p1.rows_dev = nu;
        TRY(sgemm<false, true>(p1, e1, gctas, st));
        pf.mark(P_MLP2);
        GemmShape p2 = gshape(maxU, 2 * F, F, h1, F, Lr.mlp2_w, F);
        p2.rows_dev = nu;
        TRY(sgemm<false, true>(p2, e2, gctas, st));
        pf.mark(P_MLP3);
        GemmShape p3 = gshape(maxU, 3 * F, 2 * F, h2, 2 * F, w3p(l), 2 * F);
        p3.rows_dev = nu;
        TRY(sgemm<false, true>(p3, e3, gctas, st));
        return TNET_OK;
    };
    const int ew = grid_for((int64_t)N * F, 256, sms);
    for (int l = 0; l < NL; ++l) {
        float *Xl = X + l * n9, *Xn = f32(Lw.Xn) + l * n9, *qn = f32(Lw.qn) + (int64_t)l * N * F;
        float *Y = f32(Lw.Y) + l * n9, *M = f32(Lw.M) + l * n9, *Tn = f32(Lw.Tn) + l * n9,
              *dX = f32(Lw.dX) + l * n9;
        float *Xnext = (l + 1 < NL) ? X + (l + 1) * n9 : f32(Lw.Xfin);
        pf.mark(P_NODE_ELEM);
        launch(k_node_norm, ew, 256, 0, st, Xl, N, F, qn, Xn, nbf);
        count_launch();
        TNET_LAUNCH_CHECK();
        pf.mark(P_NODE_MIX);
        if (tcm) TRY(tcg(tc::tshape_classes(N, F), Xn, nbf, 9LL * N, F, lb[l].mix1, 3 * F, F, EpiStore{Y, F, 0}));
        else TRY(sgemm<false, true>(gshape_classes(N, F, Xn, W.layer[l].mix1_w), EpiStore{Y, F, 0}, gctas, st));
        TRY(edge_mlp(l, !keep_act));
        pf.mark(P_MESSAGE);
        const float *a3l = act(Lw.a3, 3 * F, l);
#define MSG_FWD(FF)                                                                                          \
    if (tab) launch_message<FF, true>(rows_pb, atom_blocks, st, row_ptr, col, pair_of, a3l, phiu, tabfn(1 + l), Y, \
                                      N, M);                                                                 \
    else launch_message<FF, false>(rows_pb, atom_blocks, st, row_ptr, col, pair_of, a3l, phiu, tabfn(1 + l), Y, \
                                   N, M)
        if (warp_rows) launch(k_message_v4<128>, v4_blocks, 32 * kV4Warps, 0, st, row_ptr, col, pair_of, a3l, phiu, Y,
                              N, M);
        else {
            TNET_F_SWITCH(F, MSG_FWD);
        }
#undef MSG_FWD
        count_launch();
        pf.mark(P_NODE_ELEM);
        launch(k_node_update, ew, 256, 0, st, Y, M, N, F, Tn, nbf);
        count_launch();
        TNET_LAUNCH_CHECK();
        pf.mark(P_NODE_MIX);
        if (tcm) TRY(tcg(tc::tshape_classes(N, F), Tn, nbf, 9LL * N, F, lb[l].mix2, 3 * F, F, EpiStore{dX, F, 0}));
        else TRY(sgemm<false, true>(gshape_classes(N, F, Tn, W.layer[l].mix2_w), EpiStore{dX, F, 0}, gctas, st));
        pf.mark(P_NODE_ELEM);
        launch(k_residual, ew, 256, 0, st, Xn, dX, N, F, Xnext);
        count_launch();
        TNET_LAUNCH_CHECK();
    }
    float *Xfin = NL > 0 ? f32(Lw.Xfin) : X;

    // ---- output model
    pf.mark(P_OUTPUT);
    float *h = f32(Lw.h), *hn = f32(Lw.hn), *ao = f32(Lw.ao), *o = f32(Lw.o), *at = f32(Lw.at),
          *t = f32(Lw.t), *Ei = f32(Lw.Ei);
    float2 *lno = wsp<float2>(ctx, Lw.lno);
    launch(k_out_norms, N, F, 0, st, Xfin, N, F, W.out_ln_g, W.out_ln_b, h, hn, lno);
    count_launch();
    TNET_LAUNCH_CHECK();
    {
        const EpiBiasAct eo{W.out_b, ao, F, o, F, 1, nullptr};
        const EpiBiasAct eh{W.head1_b, at, H, t, H, 1, nullptr};
        if (atom_x3) {
            TRY(tcx3(tc::tshape(N, F, 3 * F), hn, N, 3 * F, wx.out, F, 3 * F, eo));
            TRY(tcx3(tc::tshape(N, H, F), o, N, F, wx.head1, H, F, eh));
        } else {
            TRY(sgemm<false, true>(gshape(N, F, 3 * F, hn, 3 * F, W.out_w, 3 * F), eo, gctas, st));
            TRY(sgemm<false, true>(gshape(N, H, F, o, F, W.head1_w, F), eh, gctas, st));
        }
    }
    launch(k_head, warps_grid, 256, 0, st, t, N, H, W.head2_w, W.head2_b, Ei);
    count_launch();
    launch(k_energy, S, 256, 0, st, Ei, sys_start, sys_end, energy);
    count_launch();
    TNET_LAUNCH_CHECK();
    if (!forces && !grad_w) return TNET_OK;

    // ---- reverse pass
    pf.mark(P_OUT_BWD);
    float *gat = f32(Lw.gat), *gao = f32(Lw.gao), *ghn = f32(Lw.ghn), *gEi = f32(Lw.gEi);
    float *gX = f32(Lw.gXa), *gdX = f32(Lw.gdX), *gTn = f32(Lw.gTn), *gM = f32(Lw.gM), *gY = f32(Lw.gY);
    float *gg = f32(Lw.gg), *ga2 = f32(Lw.ga2), *ga1 = f32(Lw.ga1), *ge = f32(Lw.ge), *gphiu = f32(Lw.gphiu);
    launch(k_head_bwd, grid_for((int64_t)N * H, 256, sms), 256, 0, st, at, N, H, W.head2_w, seed, batch, gat);
    count_launch();
    TNET_LAUNCH_CHECK();
    if (atom_x3) {
        TRY(tcx3(tc::tshape(N, F, H), gat, N, H, wx.head1T, F, H, EpiGradAct{ao, F, gao, F, 0}));
        TRY(tcx3(tc::tshape(N, 3 * F, F), gao, N, F, wx.outT, 3 * F, F, EpiStore{ghn, 3 * F, 0}, bn3));
    } else {
        TRY(sgemm<false, false>(gshape(N, F, H, gat, H, W.head1_w, F), EpiGradAct{ao, F, gao, F, 0}, gctas, st));
        TRY(sgemm<false, false>(gshape(N, 3 * F, F, gao, F, W.out_w, 3 * F), EpiStore{ghn, 3 * F, 0}, gctas, st));
    }
    launch(k_out_norms_bwd, N, F, 0, st, Xfin, h, ghn, lno, W.out_ln_g, N, F, gX);
    count_launch();
    TNET_LAUNCH_CHECK();
    if (wg) {
        launch(k_seed_atoms, (N + 255) / 256, 256, 0, st, seed, batch, N, gEi);
        count_launch();
        TNET_LAUNCH_CHECK();
        TRY(wgrad_colsum(rows1(H, 1, N, t, H, nullptr, 0, nullptr), gEi, wpart, wcap, gw(G.head2_w), 0, sms, st));
        TRY(wgrad_colsum(rows1(1, 1, N, gEi, 1, nullptr, 0, nullptr), nullptr, wpart, wcap, gw(G.head2_b), 0, sms,
                         st));
        TRY(wgrad_outer(rows1(H, F, N, gat, H, o, F, nullptr), wpart, wcap, gw(G.head1_w), 0, sms, st));
        TRY(wgrad_colsum(rows1(H, 1, N, gat, H, nullptr, 0, nullptr), nullptr, wpart, wcap, gw(G.head1_b), 0, sms,
                         st));
        TRY(wgrad_outer(rows1(F, 3 * F, N, gao, F, hn, 3 * F, nullptr), wpart, wcap, gw(G.out_w), 0, sms, st));
        TRY(wgrad_colsum(rows1(F, 1, N, gao, F, nullptr, 0, nullptr), nullptr, wpart, wcap, gw(G.out_b), 0, sms,
                         st));
        TRY(wgrad_layernorm(ghn, h, lno, N, 3 * F, wpart, wcap, gw(G.out_ln_g), sms, st));
    }
    // gphiu collects dE/dphi per pair (or, in table mode, dE/dd)
    if (NL > 0 || tab) TNET_CUDA_TRY(cudaMemsetAsync(gphiu, 0, sizeof(float) * maxU, st));
    for (int l = NL - 1; l >= 0; --l) {
        const LayerW &Lr = W.layer[l];
        const LayerW &Gr = G.layer[l];
        float *Xl = X + l * n9, *Xn = f32(Lw.Xn) + l * n9, *qn = f32(Lw.qn) + (int64_t)l * N * F;
        float *Y = f32(Lw.Y) + l * n9, *M = f32(Lw.M) + l * n9, *dX = f32(Lw.dX) + l * n9,
              *Tn = f32(Lw.Tn) + l * n9;
        pf.mark(P_NODE_BWD);
        launch(k_residual_bwd, ew, 256, 0, st, gX, dX, N, F, gdX, nbf);
        count_launch();
        TNET_LAUNCH_CHECK();
        if (tcm) TRY(tcg(tc::tshape_classes(N, F), gdX, nbf, 9LL * N, F, lb[l].mix2T, 3 * F, F, EpiStore{gTn, F, 0}));
        else TRY(sgemm<false, false>(gshape_classes(N, F, gdX, Lr.mix2_w), EpiStore{gTn, F, 0}, gctas, st));
        if (wg) TRY(wgrad_outer(rows3(gdX, Tn), wpart, wcap, gw(Gr.mix2_w), 0, sms, st));
        launch(k_T_bwd, ew, 256, 0, st, Y, M, gTn, N, F, gY, gM);
        count_launch();
        TNET_LAUNCH_CHECK();
        // this layer's radial-MLP activations: kept from the forward pass, or
        // recomputed here (same kernels, same inputs: bitwise the same values)
        if (!keep_act) TRY(edge_mlp(l, false));
        const float *a1 = act(Lw.a1, F, l), *h1 = act(Lw.h1, F, l), *a2 = act(Lw.a2, 2 * F, l),
                    *h2 = act(Lw.h2, 2 * F, l), *a3 = act(Lw.a3, 3 * F, l);
        pf.mark(P_MSG_BWD);
        // (the BF16 GEMMs read only the copy of ga3; the fp32 ga3 feeds the FP32
        // and 3xTF32 GEMMs and the weight gradients)
        float *ga3_out = (prec != 1 || wg) ? gg : nullptr;
#define MSG_BWD(FF)                                                                                          \
    launch_message_bwd<FF, false>(rows_pb, atom_blocks, st, row_ptr, col, pair_of, Y, gM, a3, phiu, tabfn(1 + l), \
                                  N, gY, nbf, ga3_out, ga3_cp, gphiu)
#define MSG_BWD_TAB(FF)                                                                                      \
    launch_message_bwd<FF, true>(rows_pb, atom_blocks, st, row_ptr, col, pair_of, Y, gM, a3, phiu, tabfn(1 + l), \
                                 N, gY, nbf, (float *)nullptr, none, gphiu)
        if (tab) {
            TNET_F_SWITCH(F, MSG_BWD_TAB);
        } else if (warp_rows) {
            if (ctx->tune[T_MSG_KERNEL] == 3)
                launch(k_message_bwd_v4<128, 3>, v4_blocks, 32 * kV4Warps, 0, st, row_ptr, col, pair_of, Y, gM, a3,
                       phiu, N, gY, nbf, ga3_out, ga3_cp, gphiu);
            else
                launch(k_message_bwd_v4<128, 2>, v4_blocks, 32 * kV4Warps, 0, st, row_ptr, col, pair_of, Y, gM, a3,
                       phiu, N, gY, nbf, ga3_out, ga3_cp, gphiu);
        } else {
            TNET_F_SWITCH(F, MSG_BWD);
        }
#undef MSG_BWD
#undef MSG_BWD_TAB
        count_launch();
        TNET_LAUNCH_CHECK();
        if (tab) {  // no radial MLP to go back through
            pf.mark(P_NODE_BWD);
            if (tcm)
                TRY(tcg(tc::tshape_classes(N, F), gY, nbf, 9LL * N, F, lb[l].mix1T, 3 * F, F, EpiStore{gX, F, 1}));
            else TRY(sgemm<false, false>(gshape_classes(N, F, gY, Lr.mix1_w), EpiStore{gX, F, 1}, gctas, st));
            launch(k_node_norm_bwd, ew, 256, 0, st, Xl, qn, N, F, gX);
            count_launch();
            TNET_LAUNCH_CHECK();
            continue;
        }
        const EpiGradAct g3{a2, 2 * F, ga2, 2 * F, 0, ga2_cp, 2 * F};
        const EpiGradAct g2{a1, F, ga1, F, 0, ga1_cp, F};
        const EpiStore g1{ge, K, l != NL - 1};
        if (tcm) {
            tc::TcShape t3 = tc::tshape(maxU, 2 * F, 3 * F), t2 = tc::tshape(maxU, F, 2 * F);
            t2.rows_dev = t3.rows_dev = nu;
            pf.mark(P_MLP3_BWD);
            TRY(tcg(t3, gg, ga3_cp, maxU, 3 * F, lb[l].mlp3T, 2 * F, 3 * F, g3, bn2));
            pf.mark(P_MLP2_BWD);
            TRY(tcg(t2, ga2, ga2_cp, maxU, 2 * F, lb[l].mlp2T, F, 2 * F, g2));
            pf.mark(P_MLP1_BWD);  // N = num_rbf: 3xTF32 in both modes
            tc::TcShape u1 = tc::tshape(maxU, K, F);
            u1.rows_dev = nu;
            TRY(tcx3(u1, ga1, maxU, F, lb[l].mlp1T, K, F, g1));
        } else {
            pf.mark(P_MLP3_BWD);
            GemmShape q3 = gshape(maxU, 2 * F, 3 * F, gg, 3 * F, w3p(l), 2 * F);
            q3.rows_dev = nu;
            TRY(sgemm<false, false>(q3, g3, gctas, st));
            pf.mark(P_MLP2_BWD);
            GemmShape q2 = gshape(maxU, F, 2 * F, ga2, 2 * F, Lr.mlp2_w, F);
            q2.rows_dev = nu;
            TRY(sgemm<false, false>(q2, g2, gctas, st));
            pf.mark(P_MLP1_BWD);
            GemmShape q1 = gshape(maxU, K, F, ga1, F, Lr.mlp1_w, K);
            q1.rows_dev = nu;
            TRY(sgemm<false, false>(q1, g1, gctas, st));
        }
        if (wg) {
            // gg is plane-major: map its rows back to the blob's c*3 + p order
            TRY(wgrad_outer(rows1(3 * F, 2 * F, maxU, gg, 3 * F, h2, 2 * F, nu), wpart, wcap, gw(Gr.mlp3_w), 0, sms, st,
                            F));
            TRY(wgrad_colsum(rows1(3 * F, 1, maxU, gg, 3 * F, nullptr, 0, nu), nullptr, wpart, wcap, gw(Gr.mlp3_b), 0,
                             sms, st, F));
            TRY(wgrad_outer(rows1(2 * F, F, maxU, ga2, 2 * F, h1, F, nu), wpart, wcap, gw(Gr.mlp2_w), 0, sms, st));
            TRY(wgrad_colsum(rows1(2 * F, 1, maxU, ga2, 2 * F, nullptr, 0, nu), nullptr, wpart, wcap, gw(Gr.mlp2_b), 0,
                             sms, st));
            TRY(wgrad_outer(rows1(F, K, maxU, ga1, F, eu, K, nu), wpart, wcap, gw(Gr.mlp1_w), 0, sms, st));
            TRY(wgrad_colsum(rows1(F, 1, maxU, ga1, F, nullptr, 0, nu), nullptr, wpart, wcap, gw(Gr.mlp1_b), 0, sms,
                             st));
            TRY(wgrad_outer(rows3(gY, Xn), wpart, wcap, gw(Gr.mix1_w), 0, sms, st));
        }
        pf.mark(P_NODE_BWD);
        if (tcm) TRY(tcg(tc::tshape_classes(N, F), gY, nbf, 9LL * N, F, lb[l].mix1T, 3 * F, F, EpiStore{gX, F, 1}));
        else TRY(sgemm<false, false>(gshape_classes(N, F, gY, Lr.mix1_w), EpiStore{gX, F, 1}, gctas, st));
        launch(k_node_norm_bwd, ew, 256, 0, st, Xl, qn, N, F, gX);
        count_launch();
        TNET_LAUNCH_CHECK();
    }
    // embedding adjoint: gX now holds dE/dX0
    pf.mark(P_EMB_NODE_BWD);
    float *gU = f32(Lw.gU), *gas2 = f32(Lw.gas2), *gas1 = f32(Lw.gas1), *gn0 = f32(Lw.gn0);
    float *gXraw = gdX;
    launch(k_emb_scale_bwd, ew, 256, 0, st, gX, Uemb, s, as2, N, F, gU, gas2, nbf);
    count_launch();
    TNET_LAUNCH_CHECK();
    if (atom_x3) {
        TRY(tcx3(tc::tshape(N, 2 * F, 3 * F), gas2, N, 3 * F, wx.emb_mlp2T, 2 * F, 3 * F,
                 EpiGradAct{as1, 2 * F, gas1, 2 * F, 0}, bn2));
        TRY(tcx3(tc::tshape(N, F, 2 * F), gas1, N, 2 * F, wx.emb_mlp1T, F, 2 * F, EpiStore{gn0, F, 0}));
    } else {
        TRY(sgemm<false, false>(gshape(N, 2 * F, 3 * F, gas2, 3 * F, W.emb_mlp2_w, 2 * F),
                                EpiGradAct{as1, 2 * F, gas1, 2 * F, 0}, gctas, st));
        TRY(sgemm<false, false>(gshape(N, F, 2 * F, gas1, 2 * F, W.emb_mlp1_w, F), EpiStore{gn0, F, 0}, gctas, st));
    }
    if (tcm) TRY(tcg(tc::tshape_classes(N, F), gU, nbf, 9LL * N, F, emixT, 3 * F, F, EpiStore{gXraw, F, 0}));
    else TRY(sgemm<false, false>(gshape_classes(N, F, gU, W.emb_mix_w), EpiStore{gXraw, F, 0}, gctas, st));
    launch(k_ln0_bwd, N, F, 0, st, Xraw, gn0, ln0, W.emb_ln_g, N, F, gXraw);
    count_launch();
    TNET_LAUNCH_CHECK();
    if (wg) {
        TRY(wgrad_outer(rows3(gU, Xraw), wpart, wcap, gw(G.emb_mix_w), 0, sms, st));
        TRY(wgrad_outer(rows1(3 * F, 2 * F, N, gas2, 3 * F, hs1, 2 * F, nullptr), wpart, wcap, gw(G.emb_mlp2_w), 0,
                        sms, st));
        TRY(wgrad_colsum(rows1(3 * F, 1, N, gas2, 3 * F, nullptr, 0, nullptr), nullptr, wpart, wcap,
                         gw(G.emb_mlp2_b), 0, sms, st));
        TRY(wgrad_outer(rows1(2 * F, F, N, gas1, 2 * F, n0, F, nullptr), wpart, wcap, gw(G.emb_mlp1_w), 0, sms, st));
        TRY(wgrad_colsum(rows1(2 * F, 1, N, gas1, 2 * F, nullptr, 0, nullptr), nullptr, wpart, wcap,
                         gw(G.emb_mlp1_b), 0, sms, st));
        TRY(wgrad_layernorm(gn0, q0, ln0, N, F, wpart, wcap, gw(G.emb_ln_g), sms, st));
    }
    pf.mark(P_EMB_EDGE_BWD);
    float *gfu = f32(Lw.gfu), *Gp = f32(Lw.gp), *gA = f32(Lw.gA_atom), *gB = f32(Lw.gB_atom);
    float4 *edge_g = wsp<float4>(ctx, Lw.edge_g);
    const int bwd_blocks = grid_for((int64_t)N * 32, 256, sms);
    // weight gradients need per-atom sums of the pair-embedding adjoints
    // (atom-parallel kernel); forces alone use the pair-parallel kernel
#define EMB_BWD(CPL)                                                                                         \
    if (wg)                                                                                                  \
        launch(k_emb_bwd<CPL>, bwd_blocks, 256, 0, st, pos, box, batch, z, row_ptr, col, pair_of, N, d.max_z, rp, \
                                                   fu, Ta, Tb, gXraw, 1, gfu, edge_g, gA, gB, gfu_cp);        \
    else if (tab)                                                                                            \
        launch(k_emb_bwd_pairs<CPL, true>, pair_grid, 256, 0, st, geo, z, uij, ue, rev, nu, N, d.max_z, fu, tf0, Ta, \
                                                            Tb, gXraw, nullptr, edge_g, none, gphiu);               \
    else                                                                                                     \
        launch(k_emb_bwd_pairs<CPL, false>, pair_grid, 256, 0, st, geo, z, uij, ue, rev, nu, N, d.max_z, fu, tf0, Ta, \
                                                             Tb, gXraw, gfu, edge_g, gfu_cp, nullptr)
    if (!wg && !tab && warp_rows)
        launch(k_emb_bwd_pairs_v4<128>, pair_grid, 256, 0, st, geo, z, uij, ue, rev, nu, N, d.max_z, fu, Ta, Tb, gXraw,
               gfu, edge_g, gfu_cp);
    else
    switch (F / 32) {
        case 2: EMB_BWD(2); break;
        case 4: EMB_BWD(4); break;
        case 6: EMB_BWD(6); break;
        case 8: EMB_BWD(8); break;
        case 10: EMB_BWD(10); break;
        case 12: EMB_BWD(12); break;
        case 14: EMB_BWD(14); break;
        case 16: EMB_BWD(16); break;
        default: return TNET_ERR_ARG;
    }
#undef EMB_BWD
    count_launch();
    TNET_LAUNCH_CHECK();
    if (!tab) {   // dE/de of the pair's radial basis also flows through the projections
        if (tcm) {
            tc::TcShape tg = tc::tshape(maxU, K, 3 * F);
            tg.rows_dev = nu;
            TRY(tcx3(tg, gfu, maxU, 3 * F, wx.dprojT, K, 3 * F, EpiStore{ge, K, NL > 0}));
        } else {
            GemmShape pg = gshape(maxU, K, 3 * F, gfu, 3 * F, W.dproj_w, K);
            pg.rows_dev = nu;
            TRY(sgemm<false, false>(pg, EpiStore{ge, K, NL > 0}, gctas, st));
        }
    }
    if (wg) {
        TRY(wgrad_outer(rows1(3 * F, K, maxU, gfu, 3 * F, eu, K, nu), wpart, wcap, gw(G.dproj_w), 0, sms, st));
        TRY(wgrad_colsum(rows1(3 * F, 1, maxU, gfu, 3 * F, nullptr, 0, nu), nullptr, wpart, wcap, gw(G.dproj_b), 0,
                         sms, st));
        const int zs = (int)Lw.zsplits;
        float *zpart = f32(Lw.zpart);
        launch(k_group_z, dim3(d.max_z, zs), F, 0, st, z, gA, gB, N, F, d.max_z, zs, zpart);
        count_launch();
        launch(k_zreduce, d.max_z, F, 0, st, zpart, zs, F, d.max_z, zpart);
        count_launch();
        launch(k_emb_tables_grad2, F + d.max_z, F, 0, st, zpart, F, d.max_z, W.emb, W.emb2_w, gw(G.emb), gw(G.emb2_w),
                                                      gw(G.emb2_b));
        count_launch();
        TNET_LAUNCH_CHECK();
    }
    if (!forces) return TNET_OK;
    pf.mark(P_FORCES);
    launch(k_pair_vec, pair_grid, 256, 0, st, pos, box, batch, uij, ue, rev, nu, rp, tab ? nullptr : ge,
           (NL > 0 && !tab) ? gphiu : nullptr, edge_g, tab ? gphiu : nullptr, Gp);
    count_launch();
    launch(k_forces, (N + 127) / 128, 128, 0, st, row_ptr, col, pair_of, Gp, N, forces);
    count_launch();
    TNET_LAUNCH_CHECK();
    return TNET_OK;
}

}  // namespace tnet
