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

namespace tnet {

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

// pair vector r_ij = mic(r_i - r_j) for rectangular boxes (box rows diagonal)
__device__ __forceinline__ void pair_vec(const float *__restrict__ pos, const float *__restrict__ box,
                                         const int32_t *__restrict__ batch, int i, int j, float &x,
                                         float &y, float &zz) {
    x = pos[3LL * i] - pos[3LL * j];
    y = pos[3LL * i + 1] - pos[3LL * j + 1];
    zz = pos[3LL * i + 2] - pos[3LL * j + 2];
    if (box) {
        const float *B = box + 9LL * (batch ? batch[i] : 0);
        x -= B[0] * rintf(x / B[0]);
        y -= B[4] * rintf(y / B[4]);
        zz -= B[8] * rintf(zz / B[8]);
    }
}

// ------------------------------------------------------- graph prep ---
// rev[e] = position of (j, i) in row j; one warp per row.
__global__ void k_rev(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int N,
                      int32_t *__restrict__ rev, int32_t *status) {
    const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (i >= N) return;
    const int lane = threadIdx.x & 31;
    for (int e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += 32) {
        const int j = col[e];
        if (j < 0 || j >= N) {
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
                up = sqrtf(x * x + y * y + zz * zz) < rc;
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
                               int2 *__restrict__ uij) {
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
                up = sqrtf(x * x + y * y + zz * zz) < rc;
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, up);
        if (e < row_ptr[i + 1] && j > i) {
            if (up) {
                const int u = base + __popc(m & ((1u << lane) - 1u));
                pair_of[e] = u;
                uij[u] = make_int2(i, j);
            } else {
                pair_of[e] = -1;
            }
        }
        base += __popc(m);
    }
}

__global__ void k_lower_assign(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                               const int32_t *__restrict__ rev, int N, int32_t *__restrict__ pair_of) {
    const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (i >= N) return;
    const int lane = threadIdx.x & 31;
    for (int e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += 32) {
        const int j = col[e];
        if (j <= i) pair_of[e] = (j == i) ? -1 : pair_of[rev[e]];
    }
}

// Radial basis and cutoff of each undirected active edge.
__global__ void k_edge_rbf(const float *__restrict__ pos, const float *__restrict__ box,
                           const int32_t *__restrict__ batch, const int2 *__restrict__ uij,
                           const int32_t *__restrict__ nu, int maxU, RadialParams rp,
                           float *__restrict__ eu, float *__restrict__ phiu) {
    const int U = *nu;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)U * rp.K;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int u = (int)(t / rp.K), k = (int)(t % rp.K);
        const int2 p = uij[u];
        float x, y, zz;
        pair_vec(pos, box, batch, p.x, p.y, x, y, zz);
        const float d = sqrtf(x * x + y * y + zz * zz);
        const float phi = cutoff_phi(d, rp);
        float e, de;
        expnorm_k(d, k, rp, phi, 0.f, e, de);
        eu[t] = e;
        if (k == 0) phiu[u] = phi;
    }
}

// Per-element pair-embedding tables: Ta[z] = W_e[:, :F] emb[z],
// Tb[z] = W_e[:, F:] emb[z] + b_e, so that Z_ij = Ta[z_i] + Tb[z_j].
__global__ void k_elem_tables(const float *__restrict__ emb, const float *__restrict__ W,
                              const float *__restrict__ b, int F, float *__restrict__ Ta,
                              float *__restrict__ Tb) {
    const int z = blockIdx.x, c = threadIdx.x;
    const float *e = emb + (int64_t)z * F;
    const float *w = W + (int64_t)c * 2 * F;
    float sa = 0.f, sb = 0.f;
    for (int k = 0; k < F; ++k) {
        sa = fmaf(w[k], e[k], sa);
        sb = fmaf(w[F + k], e[k], sb);
    }
    Ta[(int64_t)z * F + c] = sa;
    Tb[(int64_t)z * F + c] = sb + b[c];
}

// ------------------------------------------------------- embedding ---
constexpr int kEG = 4;  // edges processed per group in the embedding kernels

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
    g.d = sqrtf(x * x + y * y + zz * zz);
    g.active = (g.d < rp.rc) && (g.d > 0.f);
    const float inv = g.d > 0.f ? 1.0f / g.d : 0.f;
    g.u[0] = x * inv; g.u[1] = y * inv; g.u[2] = zz * inv;
    g.phi = g.active ? cutoff_phi(g.d, rp) : 0.f;
    g.dphi = g.active ? cutoff_dphi(g.d, rp) : 0.f;
    return g;
}

// X_raw_i = sum_j phi Z_ij (f^I I0 + f^A A0(u) + f^S S0(u)); block = F threads,
// persistent over atoms.  Dynamic smem: W [3][K][F] + e [kEG][K].
__global__ void k_emb_edges(const float *__restrict__ pos, const float *__restrict__ box,
                            const int32_t *__restrict__ batch, const int32_t *__restrict__ z,
                            const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                            int N, int F, int max_z, RadialParams rp, const float *__restrict__ dproj_w,
                            const float *__restrict__ dproj_b, const float *__restrict__ Ta,
                            const float *__restrict__ Tb, float *__restrict__ Xraw, int32_t *status) {
    extern __shared__ float sm[];
    const int K = rp.K, c = threadIdx.x;
    float *Ws = sm;                   // [3][K][F]
    float *es = Ws + 3 * K * F;       // [kEG][K]
    __shared__ EdgeGeo geo[kEG];
    for (int t = threadIdx.x; t < 3 * K * F; t += blockDim.x) {
        const int p = t / (K * F), r = t % (K * F), k = r / F, cc = r % F;
        Ws[t] = dproj_w[((int64_t)p * F + cc) * K + k];
    }
    const float bI = dproj_b[c], bA = dproj_b[F + c], bS = dproj_b[2 * F + c];
    __syncthreads();
    for (int i = blockIdx.x; i < N; i += gridDim.x) {
        int zi = z[i];
        if (zi < 0 || zi >= max_z) {
            set_status(status, TNET_ERR_Z);
            zi = 0;
        }
        const float ta = Ta[(int64_t)zi * F + c];
        float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const int e0 = row_ptr[i], e1 = row_ptr[i + 1];
        for (int eb = e0; eb < e1; eb += kEG) {
            if (threadIdx.x < kEG) {
                const int e = eb + threadIdx.x;
                if (e < e1) geo[threadIdx.x] = edge_geo(pos, box, batch, i, col[e], rp);
                else geo[threadIdx.x].active = 0;
            }
            __syncthreads();
            for (int t = threadIdx.x; t < kEG * K; t += blockDim.x) {
                const int g = t / K, k = t % K;
                float e = 0.f, de;
                if (geo[g].active) expnorm_k(geo[g].d, k, rp, geo[g].phi, 0.f, e, de);
                es[t] = e;
            }
            __syncthreads();
#pragma unroll
            for (int g = 0; g < kEG; ++g) {
                if (!geo[g].active) continue;
                float fI = bI, fA = bA, fS = bS;
                for (int k = 0; k < K; ++k) {
                    const float ek = es[g * K + k];
                    fI = fmaf(Ws[(0 * K + k) * F + c], ek, fI);
                    fA = fmaf(Ws[(1 * K + k) * F + c], ek, fA);
                    fS = fmaf(Ws[(2 * K + k) * F + c], ek, fS);
                }
                int zj = z[geo[g].j];
                zj = (zj < 0 || zj >= max_z) ? 0 : zj;
                const float pz = geo[g].phi * (ta + Tb[(int64_t)zj * F + c]);
                const float cI = pz * fI, cA = pz * fA, cS = pz * fS;
                const float ux = geo[g].u[0], uy = geo[g].u[1], uz = geo[g].u[2];
                v[0] += cI;
                v[1] += cA * ux; v[2] += cA * uy; v[3] += cA * uz;
                v[4] += cS * (ux * ux - (1.0f / 3.0f));
                v[5] += cS * (uy * uy - (1.0f / 3.0f));
                v[6] += cS * ux * uy; v[7] += cS * ux * uz; v[8] += cS * uy * uz;
            }
            __syncthreads();
        }
        store_coords(Xraw, i, c, N, F, v);
    }
}

// q0 = ||X_raw|| per channel, LayerNorm over channels -> n0; caches (mean, rstd)
__global__ void k_norm_ln(const float *__restrict__ X, int N, int F, const float *__restrict__ g,
                          const float *__restrict__ b, float *__restrict__ n0, float2 *__restrict__ ln) {
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
    if (c == 0) ln[i] = make_float2(mean, rstd);
}

// X0 = s_p * U (p = class of the coordinate), s channel-major [N][F][3]
__global__ void k_emb_scale(const float *__restrict__ U, const float *__restrict__ s, int N, int F,
                            float *__restrict__ X0) {
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
                            float *__restrict__ Xn) {
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
    }
}

// M_i = sum_j g^p_ij Y^p_j over the row (block = F threads, one atom per block)
__global__ void k_message(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                          const int32_t *__restrict__ pair_of, const float *__restrict__ gU,
                          const float *__restrict__ Y, int N, int F, float *__restrict__ M) {
    const int c = threadIdx.x;
    for (int i = blockIdx.x; i < N; i += gridDim.x) {
        float m[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int u = pair_of[e];
            if (u < 0) continue;
            const int j = col[e];
            const float *g = gU + (int64_t)u * 3 * F + 3 * c;
            const float gI = g[0], gA = g[1], gS = g[2];
            float y[9];
            load_coords(Y, j, c, N, F, y);
            m[0] = fmaf(gI, y[0], m[0]);
#pragma unroll
            for (int k = 1; k < 4; ++k) m[k] = fmaf(gA, y[k], m[k]);
#pragma unroll
            for (int k = 4; k < 9; ++k) m[k] = fmaf(gS, y[k], m[k]);
        }
        store_coords(M, i, c, N, F, m);
    }
}

// T = Y M + M Y; Tn = decomp(T) / (||T|| + 1)
__global__ void k_node_update(const float *__restrict__ Y, const float *__restrict__ M, int N, int F,
                              float *__restrict__ Tn) {
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
    }
}

// X_out = Xn + dX + dX dX
__global__ void k_residual(const float *__restrict__ Xn, const float *__restrict__ dX, int N, int F,
                           float *__restrict__ Xout) {
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
                               float *__restrict__ gdX) {
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
    }
}

// Tn = decomp(Y M + M Y) / (p + 1): gradients to Y (written) and M (written)
__global__ void k_T_bwd(const float *__restrict__ Y, const float *__restrict__ M,
                        const float *__restrict__ gTn, int N, int F, float *__restrict__ gY,
                        float *__restrict__ gM) {
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

// Message adjoint.  For atom i (block, thread per channel):
//   gY_i += sum_j g^p_ij gM_j                       (g_ij = g_ji)
//   gg[u(i,j)] = <gM_i, Y^p_j> + <gM_j, Y^p_i>       for upper edges j > i
// Each undirected entry is written once, by its upper edge: no atomics.
__global__ void k_message_bwd(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                              const int32_t *__restrict__ pair_of, const float *__restrict__ gU,
                              const float *__restrict__ Y, const float *__restrict__ gM, int N, int F,
                              float *__restrict__ gY, float *__restrict__ gg) {
    const int c = threadIdx.x;
    for (int i = blockIdx.x; i < N; i += gridDim.x) {
        float yi[9], gmi[9], acc[9];
        load_coords(Y, i, c, N, F, yi);
        load_coords(gM, i, c, N, F, gmi);
        load_coords(gY, i, c, N, F, acc);
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int u = pair_of[e];
            if (u < 0) continue;
            const int j = col[e];
            float yj[9], gmj[9];
            load_coords(gM, j, c, N, F, gmj);
            const float *g = gU + (int64_t)u * 3 * F + 3 * c;
            const float gI = g[0], gA = g[1], gS = g[2];
            acc[0] = fmaf(gI, gmj[0], acc[0]);
#pragma unroll
            for (int k = 1; k < 4; ++k) acc[k] = fmaf(gA, gmj[k], acc[k]);
#pragma unroll
            for (int k = 4; k < 9; ++k) acc[k] = fmaf(gS, gmj[k], acc[k]);
            if (j > i) {
                load_coords(Y, j, c, N, F, yj);
                float sI = gmi[0] * yj[0] + gmj[0] * yi[0];
                float sA = 0.f, sS = 0.f;
#pragma unroll
                for (int k = 1; k < 4; ++k) sA += gmi[k] * yj[k] + gmj[k] * yi[k];
#pragma unroll
                for (int k = 4; k < 9; ++k) sS += gmi[k] * yj[k] + gmj[k] * yi[k];
                float *o = gg + (int64_t)u * 3 * F + 3 * c;
                o[0] = sI; o[1] = sA; o[2] = sS;
            }
        }
        store_coords(gY, i, c, N, F, acc);
    }
}

// g = phi * silu(a3):  ga3 = gg * phi * silu'(a3) (in place), gphi += <gg, silu(a3)>
__global__ void k_mlp3_bwd(float *__restrict__ gg, const float *__restrict__ a3,
                           const float *__restrict__ phiu, const int32_t *__restrict__ nu, int W,
                           float *__restrict__ gphi) {
    const int U = *nu;
    const int lane = threadIdx.x & 31;
    for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < U;
         u += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const float phi = phiu[u];
        float s = 0.f;
        for (int n = lane; n < W; n += 32) {
            const int64_t o = u * W + n;
            const float a = a3[o], gv = gg[o];
            s = fmaf(gv, silu_f(a), s);
            gg[o] = gv * phi * silu_grad_f(a);
        }
        s = warp_sum(s);
        if (lane == 0) gphi[u] += s;
    }
}

// Xn = X / (q + 1):  gX = gXn / (q + 1) - <gXn, X> / (q + 1)^2 * dq/dX (in place)
__global__ void k_node_norm_bwd(const float *__restrict__ X, const float *__restrict__ qn, int N, int F,
                                float *__restrict__ gX) {
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
                                float *__restrict__ gU, float *__restrict__ gas2) {
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
#pragma unroll
        for (int p = 0; p < 3; ++p) gas2[t * 3 + p] = gs[p] * silu_grad_f(as2[t * 3 + p]);
    }
}

// LayerNorm of q0 = ||X_raw||: adds gq0 * dq0/dX_raw to gXraw (which holds the
// channel-mixing adjoint)
__global__ void k_ln0_bwd(const float *__restrict__ Xraw, const float *__restrict__ gn0,
                          const float2 *__restrict__ ln, const float *__restrict__ g, int N, int F,
                          float *__restrict__ gXraw) {
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

// Embedding edge adjoint and per-edge dE/dr_ij (block = F threads, persistent
// over atoms).  Also adds the radial-MLP adjoints (ge_u, gphi_u) of the
// undirected pair to its upper directed edge.  Dynamic smem:
// W [3][F][K+1] + e, de [kEG][K] + gf [kEG][3][F].
__global__ void k_emb_edges_bwd(const float *__restrict__ pos, const float *__restrict__ box,
                                const int32_t *__restrict__ batch, const int32_t *__restrict__ z,
                                const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                const int32_t *__restrict__ pair_of, int N, int F, int max_z,
                                RadialParams rp, const float *__restrict__ dproj_w,
                                const float *__restrict__ dproj_b, const float *__restrict__ Ta,
                                const float *__restrict__ Tb, const float *__restrict__ gXraw,
                                const float *__restrict__ ge_u, const float *__restrict__ gphi_u,
                                int have_mlp, float *__restrict__ gvec) {
    extern __shared__ float sm[];
    const int K = rp.K, KP = K + 1, c = threadIdx.x;
    float *Ws = sm;                    // [3][F][KP]
    float *es = Ws + 3 * F * KP;       // [kEG][K]
    float *des = es + kEG * K;         // [kEG][K]
    float *gfs = des + kEG * K;        // [kEG][3][F]
    __shared__ EdgeGeo geo[kEG];
    __shared__ float red[kEG][4][32];
    for (int t = threadIdx.x; t < 3 * F * K; t += blockDim.x) {
        const int p = t / (F * K), r = t % (F * K), cc = r / K, k = r % K;
        Ws[(p * F + cc) * KP + k] = dproj_w[t];
    }
    const float bI = dproj_b[c], bA = dproj_b[F + c], bS = dproj_b[2 * F + c];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    for (int i = blockIdx.x; i < N; i += gridDim.x) {
        int zi = z[i];
        zi = (zi < 0 || zi >= max_z) ? 0 : zi;
        const float ta = Ta[(int64_t)zi * F + c];
        float gv[9];
        load_coords(gXraw, i, c, N, F, gv);
        const int e0 = row_ptr[i], e1 = row_ptr[i + 1];
        for (int eb = e0; eb < e1; eb += kEG) {
            if (threadIdx.x < kEG) {
                const int e = eb + threadIdx.x;
                if (e < e1) geo[threadIdx.x] = edge_geo(pos, box, batch, i, col[e], rp);
                else geo[threadIdx.x].active = 0;
            }
            __syncthreads();
            for (int t = threadIdx.x; t < kEG * K; t += blockDim.x) {
                const int g = t / K, k = t % K;
                float e = 0.f, de = 0.f;
                if (geo[g].active) expnorm_k(geo[g].d, k, rp, geo[g].phi, geo[g].dphi, e, de);
                es[t] = e;
                des[t] = de;
            }
            __syncthreads();
            float part[kEG][4];
#pragma unroll
            for (int g = 0; g < kEG; ++g) {
                part[g][0] = part[g][1] = part[g][2] = part[g][3] = 0.f;
                if (!geo[g].active) {
                    gfs[(g * 3 + 0) * F + c] = 0.f;
                    gfs[(g * 3 + 1) * F + c] = 0.f;
                    gfs[(g * 3 + 2) * F + c] = 0.f;
                    continue;
                }
                float fI = bI, fA = bA, fS = bS;
                const float *wI = Ws + (0 * F + c) * KP, *wA = Ws + (1 * F + c) * KP, *wS = Ws + (2 * F + c) * KP;
                for (int k = 0; k < K; ++k) {
                    const float ek = es[g * K + k];
                    fI = fmaf(wI[k], ek, fI);
                    fA = fmaf(wA[k], ek, fA);
                    fS = fmaf(wS[k], ek, fS);
                }
                int zj = z[geo[g].j];
                zj = (zj < 0 || zj >= max_z) ? 0 : zj;
                const float Z = ta + Tb[(int64_t)zj * F + c];
                const float phi = geo[g].phi;
                const float ux = geo[g].u[0], uy = geo[g].u[1], uz = geo[g].u[2];
                const float cA = phi * Z * fA, cS = phi * Z * fS;
                const float gcI = gv[0];
                const float gcA = gv[1] * ux + gv[2] * uy + gv[3] * uz;
                const float bxx = ux * ux - (1.0f / 3.0f), byy = uy * uy - (1.0f / 3.0f);
                const float gcS = gv[4] * bxx + gv[5] * byy + gv[6] * ux * uy + gv[7] * ux * uz + gv[8] * uy * uz;
                part[g][0] = Z * (gcI * fI + gcA * fA + gcS * fS);  // d/dphi
                part[g][1] = cA * gv[1] + cS * (2.f * ux * gv[4] + uy * gv[6] + uz * gv[7]);
                part[g][2] = cA * gv[2] + cS * (2.f * uy * gv[5] + ux * gv[6] + uz * gv[8]);
                part[g][3] = cA * gv[3] + cS * (ux * gv[7] + uy * gv[8]);
                const float pz = phi * Z;
                gfs[(g * 3 + 0) * F + c] = gcI * pz;
                gfs[(g * 3 + 1) * F + c] = gcA * pz;
                gfs[(g * 3 + 2) * F + c] = gcS * pz;
            }
#pragma unroll
            for (int g = 0; g < kEG; ++g)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float s = warp_sum(part[g][q]);
                    if (lane == 0) red[g][q][wid] = s;
                }
            __syncthreads();
            // warp g: dE/dd of edge g = sum_k (ge_k de_k/dd) + gphi dphi/dd
            for (int g = wid; g < kEG; g += nw) {
                float s = 0.f;
                if (geo[g].active) {
                    const int e = eb + g;
                    const int u = have_mlp ? pair_of[e] : -1;
                    const bool upper = (u >= 0) && (geo[g].j > i);
                    for (int k = lane; k < K; k += 32) {
                        float gek = 0.f;
                        for (int p = 0; p < 3; ++p) {
                            const float *gf = gfs + (g * 3 + p) * F;
                            const float *w = Ws + p * F * KP + k;
                            for (int cc = 0; cc < F; ++cc) gek = fmaf(gf[cc], w[cc * KP], gek);
                        }
                        if (upper) gek += ge_u[(int64_t)u * K + k];
                        s = fmaf(gek, des[g * K + k], s);
                    }
                    s = warp_sum(s);
                    if (lane == 0) {
                        float gphi = 0.f, gux = 0.f, guy = 0.f, guz = 0.f;
                        for (int w = 0; w < nw; ++w) {
                            gphi += red[g][0][w];
                            gux += red[g][1][w];
                            guy += red[g][2][w];
                            guz += red[g][3][w];
                        }
                        if (upper) gphi += gphi_u[u];
                        const float gd = s + gphi * geo[g].dphi;
                        const float ux = geo[g].u[0], uy = geo[g].u[1], uz = geo[g].u[2];
                        const float dot = gux * ux + guy * uy + guz * uz;
                        const float inv = 1.0f / geo[g].d;
                        float *o = gvec + 3LL * e;
                        o[0] = gd * ux + (gux - dot * ux) * inv;
                        o[1] = gd * uy + (guy - dot * uy) * inv;
                        o[2] = gd * uz + (guz - dot * uz) * inv;
                    }
                } else if (lane == 0 && eb + g < e1) {
                    float *o = gvec + 3LL * (eb + g);
                    o[0] = o[1] = o[2] = 0.f;
                }
            }
            __syncthreads();
        }
    }
}

// F_i = -sum_{e in row i} (gvec[e] - gvec[rev[e]]) over the active edges of
// the row, summed in row order by one thread per atom so the result does not
// depend on inactive (skin) entries of the list.
__global__ void k_forces(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ rev,
                         const int32_t *__restrict__ pair_of, const float *__restrict__ gvec, int N,
                         float *__restrict__ forces) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        if (pair_of[e] < 0) continue;
        const int r = rev[e];
        fx += gvec[3LL * e] - gvec[3LL * r];
        fy += gvec[3LL * e + 1] - gvec[3LL * r + 1];
        fz += gvec[3LL * e + 2] - gvec[3LL * r + 2];
    }
    forces[3LL * i] = -fx;
    forces[3LL * i + 1] = -fy;
    forces[3LL * i + 2] = -fz;
}

// Opt the kernels with large dynamic shared memory into it (once per context).
int tnet_kernel_setup(tnet_ctx *c) {
    const int F = c->d.F, K = c->d.K;
    const size_t fwd = sizeof(float) * (3 * K * F + kEG * K);
    const size_t bwd = sizeof(float) * (3 * F * (K + 1) + 2 * kEG * K + kEG * 3 * F);
    TNET_CUDA_TRY(cudaFuncSetAttribute(k_emb_edges, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd));
    TNET_CUDA_TRY(cudaFuncSetAttribute(k_emb_edges_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd));
    return TNET_OK;
}

// ============================================================ driver ===
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

int energy_forces_impl(tnet_ctx *ctx, const float *wblob, int N, int S, const int32_t *z,
                       const float *pos, const int32_t *batch, const float *box,
                       const int32_t *row_ptr, const int32_t *col, const float *seed,
                       double *energy, float *forces, float *grad_w, int32_t *status,
                       cudaStream_t st) {
    if (grad_w) return TNET_ERR_UNSUPPORTED;
    const tnet_model_desc &d = ctx->d;
    const Layout &Lw = ctx->lay;
    const int F = d.F, K = d.K, NL = d.L, H = F / 2;
    const int sms = ctx->num_sms;
    const RadialParams rp = ctx->rp;
    Weights W;
    weight_offsets(&d, wblob, &W);
    auto f32 = [&](size_t off) { return wsp<float>(ctx, off); };
    auto i32 = [&](size_t off) { return wsp<int32_t>(ctx, off); };
    const int64_t n9 = Lw.node9;
    const int maxU = (int)Lw.maxU;
    int32_t *sys_start = i32(Lw.sys_start), *sys_end = i32(Lw.sys_end);
    int32_t *rev = i32(Lw.rev), *pair_of = i32(Lw.pair_of), *ucnt = i32(Lw.ucnt);
    int32_t *nu = i32(Lw.nu);
    int2 *uij = wsp<int2>(ctx, Lw.uedge);
    float *Ta = f32(Lw.Ta), *Tb = f32(Lw.Tb);
    const int warps_grid = (int)(((int64_t)N * 32 + 255) / 256);

    // ---- graph prep
    ProfSeq pf(ctx, st);
    pf.mark(P_PREP);
    TNET_CUDA_TRY(cudaMemsetAsync(sys_start, 0, sizeof(int32_t) * S, st));
    TNET_CUDA_TRY(cudaMemsetAsync(sys_end, 0, sizeof(int32_t) * S, st));
    if (N > 0) TRY(sys_bounds(batch, N, S, sys_start, sys_end, status, st));
    if (N > 0) {
        k_rev<<<warps_grid, 256, 0, st>>>(row_ptr, col, N, rev, status);
        count_launch();
        k_upper_count<<<warps_grid, 256, 0, st>>>(pos, box, batch, row_ptr, col, N, rp.rc, ucnt);
        count_launch();
        TNET_LAUNCH_CHECK();
    }
    TRY(scan_exclusive_i32(ucnt, ucnt, N, i32(Lw.scan_tmp), nu, nullptr, st));
    if (N > 0) {
        k_upper_assign<<<warps_grid, 256, 0, st>>>(pos, box, batch, row_ptr, col, N, rp.rc, ucnt,
                                                   pair_of, uij);
        count_launch();
        k_lower_assign<<<warps_grid, 256, 0, st>>>(row_ptr, col, rev, N, pair_of);
        count_launch();
        TNET_LAUNCH_CHECK();
    }
    float *eu = f32(Lw.eu), *phiu = f32(Lw.phiu);
    k_edge_rbf<<<sms * 8, 256, 0, st>>>(pos, box, batch, uij, nu, maxU, rp, eu, phiu);
    count_launch();
    k_elem_tables<<<d.max_z, F, 0, st>>>(W.emb, W.emb2_w, W.emb2_b, F, Ta, Tb);
    count_launch();
    TNET_LAUNCH_CHECK();

    // ---- embedding
    pf.mark(P_EMB_EDGE);
    float *Xraw = f32(Lw.Xraw), *Uemb = f32(Lw.Uemb), *n0 = f32(Lw.n0), *as1 = f32(Lw.as1),
          *hs1 = f32(Lw.hs1), *as2 = f32(Lw.as2), *s = f32(Lw.s);
    float2 *ln0 = wsp<float2>(ctx, Lw.ln0);
    const int emb_blocks = N < sms * 4 ? (N > 0 ? N : 1) : sms * 4;
    const size_t emb_smem = sizeof(float) * (3 * K * F + kEG * K);
    if (N > 0) {
        k_emb_edges<<<emb_blocks, F, emb_smem, st>>>(pos, box, batch, z, row_ptr, col, N, F, d.max_z, rp,
                                                     W.dproj_w, W.dproj_b, Ta, Tb, Xraw, status);
        count_launch();
        k_norm_ln<<<N, F, 0, st>>>(Xraw, N, F, W.emb_ln_g, W.emb_ln_b, n0, ln0);
        count_launch();
        TNET_LAUNCH_CHECK();
    }
    pf.mark(P_EMB_NODE);
    TRY(sgemm<false, true>(gshape(N, 2 * F, F, n0, F, W.emb_mlp1_w, F),
                           EpiBiasAct{W.emb_mlp1_b, as1, 2 * F, hs1, 2 * F, 1, nullptr}, sms, st));
    TRY(sgemm<false, true>(gshape(N, 3 * F, 2 * F, hs1, 2 * F, W.emb_mlp2_w, 2 * F),
                           EpiBiasAct{W.emb_mlp2_b, as2, 3 * F, s, 3 * F, 1, nullptr}, sms, st));
    TRY(sgemm<false, true>(gshape_classes(N, F, Xraw, W.emb_mix_w), EpiStore{Uemb, F, 0}, sms, st));
    float *X = f32(Lw.Xin);  // layer 0 input
    k_emb_scale<<<grid_for((int64_t)N * F, 256, sms), 256, 0, st>>>(Uemb, s, N, F, X);
    count_launch();
    TNET_LAUNCH_CHECK();

    // ---- interaction layers
    float *a1 = f32(Lw.a1), *h1 = f32(Lw.h1), *a2 = f32(Lw.a2), *h2 = f32(Lw.h2), *a3 = f32(Lw.a3),
          *gbuf = f32(Lw.g);
    auto edge_mlp = [&](int l) -> int {
        const LayerW &Lr = W.layer[l];
        pf.mark(P_MLP1);
        GemmShape p1 = gshape(maxU, F, K, eu, K, Lr.mlp1_w, K);
        p1.rows_dev = nu;
        TRY(sgemm<false, true>(p1, EpiBiasAct{Lr.mlp1_b, a1, F, h1, F, 1, nullptr}, sms, st));
        pf.mark(P_MLP2);
        GemmShape p2 = gshape(maxU, 2 * F, F, h1, F, Lr.mlp2_w, F);
        p2.rows_dev = nu;
        TRY(sgemm<false, true>(p2, EpiBiasAct{Lr.mlp2_b, a2, 2 * F, h2, 2 * F, 1, nullptr}, sms, st));
        pf.mark(P_MLP3);
        GemmShape p3 = gshape(maxU, 3 * F, 2 * F, h2, 2 * F, Lr.mlp3_w, 2 * F);
        p3.rows_dev = nu;
        TRY(sgemm<false, true>(p3, EpiBiasAct{Lr.mlp3_b, a3, 3 * F, gbuf, 3 * F, 1, phiu}, sms, st));
        return TNET_OK;
    };
    const int ew = grid_for((int64_t)N * F, 256, sms);
    const int atom_blocks = N < sms * 8 ? (N > 0 ? N : 1) : sms * 8;
    for (int l = 0; l < NL; ++l) {
        float *Xl = X + l * n9, *Xn = f32(Lw.Xn) + l * n9, *qn = f32(Lw.qn) + (int64_t)l * N * F;
        float *Y = f32(Lw.Y) + l * n9, *M = f32(Lw.M) + l * n9, *Tn = f32(Lw.Tn) + l * n9,
              *dX = f32(Lw.dX) + l * n9;
        float *Xnext = (l + 1 < NL) ? X + (l + 1) * n9 : f32(Lw.Xfin);
        pf.mark(P_NODE_ELEM);
        k_node_norm<<<ew, 256, 0, st>>>(Xl, N, F, qn, Xn);
        count_launch();
        TNET_LAUNCH_CHECK();
        pf.mark(P_NODE_MIX);
        TRY(sgemm<false, true>(gshape_classes(N, F, Xn, W.layer[l].mix1_w), EpiStore{Y, F, 0}, sms, st));
        TRY(edge_mlp(l));
        pf.mark(P_MESSAGE);
        k_message<<<atom_blocks, F, 0, st>>>(row_ptr, col, pair_of, gbuf, Y, N, F, M);
        count_launch();
        pf.mark(P_NODE_ELEM);
        k_node_update<<<ew, 256, 0, st>>>(Y, M, N, F, Tn);
        count_launch();
        TNET_LAUNCH_CHECK();
        pf.mark(P_NODE_MIX);
        TRY(sgemm<false, true>(gshape_classes(N, F, Tn, W.layer[l].mix2_w), EpiStore{dX, F, 0}, sms, st));
        pf.mark(P_NODE_ELEM);
        k_residual<<<ew, 256, 0, st>>>(Xn, dX, N, F, Xnext);
        count_launch();
        TNET_LAUNCH_CHECK();
    }
    float *Xfin = NL > 0 ? f32(Lw.Xfin) : X;

    // ---- output model
    pf.mark(P_OUTPUT);
    float *h = f32(Lw.h), *hn = f32(Lw.hn), *ao = f32(Lw.ao), *o = f32(Lw.o), *at = f32(Lw.at),
          *t = f32(Lw.t), *Ei = f32(Lw.Ei);
    float2 *lno = wsp<float2>(ctx, Lw.lno);
    if (N > 0) {
        k_out_norms<<<N, F, 0, st>>>(Xfin, N, F, W.out_ln_g, W.out_ln_b, h, hn, lno);
        count_launch();
        TNET_LAUNCH_CHECK();
    }
    TRY(sgemm<false, true>(gshape(N, F, 3 * F, hn, 3 * F, W.out_w, 3 * F),
                           EpiBiasAct{W.out_b, ao, F, o, F, 1, nullptr}, sms, st));
    TRY(sgemm<false, true>(gshape(N, H, F, o, F, W.head1_w, F),
                           EpiBiasAct{W.head1_b, at, H, t, H, 1, nullptr}, sms, st));
    if (N > 0) {
        k_head<<<warps_grid, 256, 0, st>>>(t, N, H, W.head2_w, W.head2_b, Ei);
        count_launch();
    }
    k_energy<<<S, 256, 0, st>>>(Ei, sys_start, sys_end, energy);
    count_launch();
    TNET_LAUNCH_CHECK();
    if (!forces || N == 0) return TNET_OK;

    // ---- reverse pass
    pf.mark(P_OUT_BWD);
    float *gat = f32(Lw.gat), *gao = f32(Lw.gao), *ghn = f32(Lw.ghn);
    float *gX = f32(Lw.gXa), *gdX = f32(Lw.gdX), *gTn = f32(Lw.gTn), *gM = f32(Lw.gM), *gY = f32(Lw.gY);
    float *gg = f32(Lw.gg), *ga2 = f32(Lw.ga2), *ga1 = f32(Lw.ga1), *ge = f32(Lw.ge), *gphiu = f32(Lw.gphiu);
    k_head_bwd<<<grid_for((int64_t)N * H, 256, sms), 256, 0, st>>>(at, N, H, W.head2_w, seed, batch, gat);
    count_launch();
    TNET_LAUNCH_CHECK();
    TRY(sgemm<false, false>(gshape(N, F, H, gat, H, W.head1_w, F), EpiGradAct{ao, F, gao, F, 0}, sms, st));
    TRY(sgemm<false, false>(gshape(N, 3 * F, F, gao, F, W.out_w, 3 * F), EpiStore{ghn, 3 * F, 0}, sms, st));
    k_out_norms_bwd<<<N, F, 0, st>>>(Xfin, h, ghn, lno, W.out_ln_g, N, F, gX);
    count_launch();
    TNET_LAUNCH_CHECK();
    if (NL > 0) TNET_CUDA_TRY(cudaMemsetAsync(gphiu, 0, sizeof(float) * maxU, st));
    for (int l = NL - 1; l >= 0; --l) {
        const LayerW &Lr = W.layer[l];
        float *Xl = X + l * n9, *Xn = f32(Lw.Xn) + l * n9, *qn = f32(Lw.qn) + (int64_t)l * N * F;
        float *Y = f32(Lw.Y) + l * n9, *M = f32(Lw.M) + l * n9, *dX = f32(Lw.dX) + l * n9;
        (void)Xn;
        pf.mark(P_NODE_BWD);
        k_residual_bwd<<<ew, 256, 0, st>>>(gX, dX, N, F, gdX);
        count_launch();
        TNET_LAUNCH_CHECK();
        TRY(sgemm<false, false>(gshape_classes(N, F, gdX, Lr.mix2_w), EpiStore{gTn, F, 0}, sms, st));
        k_T_bwd<<<ew, 256, 0, st>>>(Y, M, gTn, N, F, gY, gM);
        count_launch();
        TNET_LAUNCH_CHECK();
        TRY(edge_mlp(l));  // recompute a1, h1, a2, h2, a3, g of this layer
        pf.mark(P_MSG_BWD);
        k_message_bwd<<<atom_blocks, F, 0, st>>>(row_ptr, col, pair_of, gbuf, Y, gM, N, F, gY, gg);
        count_launch();
        pf.mark(P_MLP_ELEM_BWD);
        k_mlp3_bwd<<<sms * 8, 256, 0, st>>>(gg, a3, phiu, nu, 3 * F, gphiu);
        count_launch();
        TNET_LAUNCH_CHECK();
        pf.mark(P_MLP3_BWD);
        GemmShape q3 = gshape(maxU, 2 * F, 3 * F, gg, 3 * F, Lr.mlp3_w, 2 * F);
        q3.rows_dev = nu;
        TRY(sgemm<false, false>(q3, EpiGradAct{a2, 2 * F, ga2, 2 * F, 0}, sms, st));
        pf.mark(P_MLP2_BWD);
        GemmShape q2 = gshape(maxU, F, 2 * F, ga2, 2 * F, Lr.mlp2_w, F);
        q2.rows_dev = nu;
        TRY(sgemm<false, false>(q2, EpiGradAct{a1, F, ga1, F, 0}, sms, st));
        pf.mark(P_MLP1_BWD);
        GemmShape q1 = gshape(maxU, K, F, ga1, F, Lr.mlp1_w, K);
        q1.rows_dev = nu;
        TRY(sgemm<false, false>(q1, EpiStore{ge, K, l != NL - 1}, sms, st));
        pf.mark(P_NODE_BWD);
        TRY(sgemm<false, false>(gshape_classes(N, F, gY, Lr.mix1_w), EpiStore{gX, F, 1}, sms, st));
        k_node_norm_bwd<<<ew, 256, 0, st>>>(Xl, qn, N, F, gX);
        count_launch();
        TNET_LAUNCH_CHECK();
    }
    // embedding adjoint: gX now holds dE/dX0
    pf.mark(P_EMB_NODE_BWD);
    float *gU = f32(Lw.gU), *gas2 = f32(Lw.gas2), *gas1 = f32(Lw.gas1), *gn0 = f32(Lw.gn0);
    float *gXraw = gdX;
    k_emb_scale_bwd<<<ew, 256, 0, st>>>(gX, Uemb, s, as2, N, F, gU, gas2);
    count_launch();
    TNET_LAUNCH_CHECK();
    TRY(sgemm<false, false>(gshape(N, 2 * F, 3 * F, gas2, 3 * F, W.emb_mlp2_w, 2 * F),
                            EpiGradAct{as1, 2 * F, gas1, 2 * F, 0}, sms, st));
    TRY(sgemm<false, false>(gshape(N, F, 2 * F, gas1, 2 * F, W.emb_mlp1_w, F), EpiStore{gn0, F, 0}, sms, st));
    TRY(sgemm<false, false>(gshape_classes(N, F, gU, W.emb_mix_w), EpiStore{gXraw, F, 0}, sms, st));
    k_ln0_bwd<<<N, F, 0, st>>>(Xraw, gn0, ln0, W.emb_ln_g, N, F, gXraw);
    count_launch();
    TNET_LAUNCH_CHECK();
    pf.mark(P_EMB_EDGE_BWD);
    float *gvec = f32(Lw.gvec);
    const size_t bwd_smem = sizeof(float) * (3 * F * (K + 1) + 2 * kEG * K + kEG * 3 * F);
    k_emb_edges_bwd<<<emb_blocks, F, bwd_smem, st>>>(pos, box, batch, z, row_ptr, col, pair_of, N, F,
                                                     d.max_z, rp, W.dproj_w, W.dproj_b, Ta, Tb, gXraw,
                                                     ge, gphiu, NL > 0, gvec);
    count_launch();
    pf.mark(P_FORCES);
    k_forces<<<(N + 127) / 128, 128, 0, st>>>(row_ptr, rev, pair_of, gvec, N, forces);
    count_launch();
    TNET_LAUNCH_CHECK();
    return TNET_OK;
}

}  // namespace tnet
