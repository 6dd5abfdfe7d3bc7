// Cell-list neighbor search (Sec. 2.5.1) and device-wide exclusive scans.
//
// Differences from the paper's engine, by design: one cell list per system
// (cells keyed by (system, cell)) instead of a single list for the whole
// batch, so systems never test each other's atoms (the paper notes its
// shared list degrades with batch size); the output is a receiver-sorted
// CSR with ascending columns and an exact count instead of a -1 padded pair
// list; overflow is reported in a device status word with the needed size.
#include "internal.cuh"

namespace tnet {

// ------------------------------------------------------------------ scan ---
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t *total, int32_t *smem) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int32_t w = lane < (int)(blockDim.x >> 5) ? smem[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        smem[lane] = w;  // inclusive warp prefix
    }
    __syncthreads();
    const int32_t warp_excl = wid ? smem[wid - 1] : 0;
    *total = smem[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_excl + x - v;
}

__global__ void k_scan_tiles(const int32_t *__restrict__ in, int32_t *__restrict__ out, int n,
                             int32_t *__restrict__ tile_sums, const int32_t *__restrict__ gate) {
    pdl_entry();
    if (gate && *gate == 0) return;  // gated rebuild: nothing to do
    __shared__ int32_t sm[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        sum += v[k];
    }
    int32_t total;
    int32_t run = block_exclusive_scan(sum, &total, sm);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// single block: exclusive scan of the tile sums (nt <= kScanTile)
__global__ void k_scan_top(int32_t *__restrict__ tile_sums, int nt, int32_t *__restrict__ grand,
                           const int32_t *__restrict__ gate) {
    pdl_entry();
    if (gate && *gate == 0) return;  // gated rebuild: nothing to do
    __shared__ int32_t sm[32];
    const int base = threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < nt) ? tile_sums[base + k] : 0;
        sum += v[k];
    }
    int32_t total;
    int32_t run = block_exclusive_scan(sum, &total, sm);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < nt) tile_sums[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) *grand = total;
}

__global__ void k_scan_add(int32_t *__restrict__ out, int n, const int32_t *__restrict__ tile_sums,
                           const int32_t *__restrict__ grand, int32_t *__restrict__ total_dev,
                           int64_t *__restrict__ total64_dev, const int32_t *__restrict__ gate) {
    pdl_entry();
    if (gate && *gate == 0) return;  // gated rebuild: nothing to do
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_sums[i / kScanTile];
    if (i == 0) {
        out[n] = *grand;
        if (total_dev) *total_dev = *grand;
        if (total64_dev) *total64_dev = *grand;
    }
}

// out[0..n] = exclusive scan of in[0..n), out[n] = total.  tmp needs
// ceil(n / 4096) + 1 ints.  n <= 4096 * 4096.
// dst[0..n) = 0 unless a gate is given and clear (the gated form of a memset)
__global__ void k_zero_i32(int32_t *__restrict__ dst, int64_t n, const int32_t *__restrict__ gate) {
    pdl_entry();
    if (gate && *gate == 0) return;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = 0;
}

int scan_exclusive_i32(const int32_t *in, int32_t *out, int n, int32_t *tmp, int32_t *total_dev,
                       int64_t *total64_dev, cudaStream_t st, const int32_t *gate) {
    const int nt = (n + kScanTile - 1) / kScanTile;
    if (nt > kScanTile) return TNET_ERR_ARG;
    const int ntl = nt > 0 ? nt : 1;
    if (n > 0) {
        launch(k_scan_tiles, nt, kScanThreads, 0, st, in, out, n, tmp, gate);
        count_launch();
    }
    else if (gate) {
        launch(k_zero_i32, 1, 32, 0, st, tmp, 1, gate);
        count_launch();
    } else TNET_CUDA_TRY(cudaMemsetAsync(tmp, 0, sizeof(int32_t), st));
    launch(k_scan_top, 1, kScanThreads, 0, st, tmp, ntl, tmp + ntl, gate);
    count_launch();
    launch(k_scan_add, (n + 255) / 256 + 1, 256, 0, st, out, n, tmp, tmp + ntl, total_dev, total64_dev, gate);
    count_launch();
    TNET_LAUNCH_CHECK();
    return TNET_OK;
}

// --------------------------------------------------------------- systems ---
__global__ void k_sys_bounds(const int32_t *__restrict__ batch, int N, int S,
                             int32_t *__restrict__ sys_start, int32_t *__restrict__ sys_end,
                             int32_t *status, const int32_t *__restrict__ gate) {
    pdl_entry();
    if (gate && *gate == 0) return;  // gated rebuild: nothing to do
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int b = batch ? batch[n] : 0;
    if (b < 0 || b >= S) {
        set_status(status, TNET_ERR_ARG);
        return;
    }
    const int bp = (n > 0) ? (batch ? batch[n - 1] : 0) : -1;
    const int bn = (n + 1 < N) ? (batch ? batch[n + 1] : 0) : S;
    if (bp > b) set_status(status, TNET_ERR_ARG);  // not sorted
    if (bp != b) sys_start[b] = n;
    if (bn != b) sys_end[b] = n + 1;
}

int sys_bounds(const int32_t *batch, int N, int S, int32_t *sys_start, int32_t *sys_end,
               int32_t *status, cudaStream_t st) {
    launch(k_sys_bounds, (N + 255) / 256, 256, 0, st, batch, N, S, sys_start, sys_end, status, nullptr);
    count_launch();
    TNET_LAUNCH_CHECK();
    return TNET_OK;
}

// One block per system: bounding box, finiteness, box checks and cell grid.
__global__ void k_sys_setup(const float *__restrict__ pos, const float *__restrict__ box, float cutoff,
                            const int32_t *__restrict__ sys_start, const int32_t *__restrict__ sys_end,
                            SysInfo *__restrict__ info, int32_t *__restrict__ ncell, int32_t *status,
                            const int32_t *__restrict__ gate) {
    pdl_entry();
    if (gate && *gate == 0) return;  // gated rebuild: nothing to do
    const int s = blockIdx.x;
    const int a0 = sys_start[s], a1 = sys_end[s];
    float lo[3] = {3.4e38f, 3.4e38f, 3.4e38f}, hi[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
    int bad = 0;
    for (int n = a0 + threadIdx.x; n < a1; n += blockDim.x) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float x = pos[3LL * n + k];
            if (!isfinite(x)) bad = 1;
            lo[k] = fminf(lo[k], x);
            hi[k] = fmaxf(hi[k], x);
        }
    }
    __shared__ float slo[3][32], shi[3][32];
    __shared__ int sbad;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    if (bad) atomicOr(&sbad, 1);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float l = lo[k], h = hi[k];
        for (int o = 16; o; o >>= 1) {
            l = fminf(l, __shfl_xor_sync(0xffffffffu, l, o));
            h = fmaxf(h, __shfl_xor_sync(0xffffffffu, h, o));
        }
        if (lane == 0) {
            slo[k][wid] = l;
            shi[k][wid] = h;
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const int nw = blockDim.x >> 5;
    for (int k = 0; k < 3; ++k) {
        for (int w = 1; w < nw; ++w) {
            slo[k][0] = fminf(slo[k][0], slo[k][w]);
            shi[k][0] = fmaxf(shi[k][0], shi[k][w]);
        }
    }
    SysInfo si;
    const int na = a1 - a0;
    if (sbad) set_status(status, TNET_ERR_NAN);
    if (box) {
        // rows a = (ax,0,0), b = (bx,by,0), c = (cx,cy,cz): rectangular or
        // triclinic.  Cells are cut along a, b, c in fractional coordinates,
        // nc_k = floor(w_k / cutoff) of them, where w_k is the perpendicular
        // width between the box faces spanned by the other two vectors: the
        // planes between cells are then >= cutoff apart, so a pair within
        // the cutoff is in the same or an adjacent cell along every axis
        // (with a 1e-4 relative slack, so rounding at a cell face never
        // matters).
        const float *B = box + 9LL * s;
        si.pbc = 1;
        const double ax = B[0], bx = B[3], by = B[4], cx = B[6], cy = B[7], cz = B[8];
        if (B[1] != 0.f || B[2] != 0.f || B[5] != 0.f || !(ax > 0.0) || !(by > 0.0) || !(cz > 0.0))
            set_status(status, TNET_ERR_BOX);
        const double n0 = by * cz, n1 = -bx * cz, n2 = bx * cy - by * cx;  // b x c
        const double w[3] = {ax * by * cz / sqrt(n0 * n0 + n1 * n1 + n2 * n2), by * cz / sqrt(cz * cz + cy * cy),
                             cz};
        si.L[0] = (float)ax; si.L[1] = (float)by; si.L[2] = (float)cz;
        si.tilt[0] = (float)bx; si.tilt[1] = (float)cx; si.tilt[2] = (float)cy;
        for (int k = 0; k < 3; ++k) {
            if (!(w[k] >= 2.0 * cutoff)) set_status(status, TNET_ERR_BOX);
            si.origin[k] = 0.f;
            const int nc = (w[k] > 0.0 && w[k] < 1e30) ? (int)floor(w[k] / (cutoff * 1.0001)) : 1;
            si.nc[k] = nc < 1 ? 1 : nc;
        }
    } else {
        si.pbc = 0;
        for (int k = 0; k < 3; ++k) {
            si.L[k] = 0.f;
            si.tilt[k] = 0.f;
            const float ext = na > 0 ? (shi[k][0] - slo[k][0]) : 0.f;
            si.origin[k] = na > 0 ? slo[k][0] : 0.f;
            int nc = (ext > 0.f && isfinite(ext)) ? (int)floorf(ext / cutoff) : 1;
            si.nc[k] = nc < 1 ? 1 : (nc > 1024 ? 1024 : nc);
        }
    }
    // keep the grid no finer than ~2 cells per atom (cells only get wider)
    const int64_t budget = 2LL * na + 8;
    while ((int64_t)si.nc[0] * si.nc[1] * si.nc[2] > budget) {
        int k = 0;
        if (si.nc[1] > si.nc[k]) k = 1;
        if (si.nc[2] > si.nc[k]) k = 2;
        si.nc[k] = si.nc[k] / 2 > 1 ? si.nc[k] / 2 : 1;
    }
    for (int k = 0; k < 3; ++k) {  // (PBC: cells per unit of fractional coordinate)
        const float width = si.pbc ? 1.0f : (na > 0 ? shi[k][0] - slo[k][0] : 0.f);
        si.inv_cell[k] = width > 0.f ? si.nc[k] / width : 0.f;
    }
    si.cell_off = 0;
    si.pad = 0;
    info[s] = si;
    ncell[s] = na > 0 ? si.nc[0] * si.nc[1] * si.nc[2] : 0;
}

__device__ __forceinline__ int cell_index(float u, int nc) {
    int c = (int)floorf(u);
    c = c < 0 ? 0 : c;
    return c >= nc ? nc - 1 : c;
}
// Cell of a point.  Without PBC: along x, y, z from the grid's corner.  With
// PBC: along a, b, c from the fractional coordinates (back substitution in
// the lower-triangular box, wrapped into [0, 1)).  Fixed rounding, so the
// binning pass and the pair passes put an atom in the same cell.
__device__ __forceinline__ void point_cell(float x, float y, float z, const SysInfo &s, int &ca, int &cb, int &cc) {
    if (s.pbc) {
        const float fc = __fdiv_rn(z, s.L[2]);
        const float fb = __fdiv_rn(__fsub_rn(y, __fmul_rn(fc, s.tilt[2])), s.L[1]);
        const float fa = __fdiv_rn(__fsub_rn(__fsub_rn(x, __fmul_rn(fc, s.tilt[1])), __fmul_rn(fb, s.tilt[0])),
                                   s.L[0]);
        ca = cell_index(__fmul_rn(__fsub_rn(fa, floorf(fa)), s.inv_cell[0]), s.nc[0]);
        cb = cell_index(__fmul_rn(__fsub_rn(fb, floorf(fb)), s.inv_cell[1]), s.nc[1]);
        cc = cell_index(__fmul_rn(__fsub_rn(fc, floorf(fc)), s.inv_cell[2]), s.nc[2]);
    } else {
        ca = cell_index(__fmul_rn(__fsub_rn(x, s.origin[0]), s.inv_cell[0]), s.nc[0]);
        cb = cell_index(__fmul_rn(__fsub_rn(y, s.origin[1]), s.inv_cell[1]), s.nc[1]);
        cc = cell_index(__fmul_rn(__fsub_rn(z, s.origin[2]), s.inv_cell[2]), s.nc[2]);
    }
}

__global__ void k_bin(const float *__restrict__ pos, const int32_t *__restrict__ batch, int N,
                      const SysInfo *__restrict__ info, const int32_t *__restrict__ cell_off,
                      int32_t *__restrict__ cell_of, int32_t *__restrict__ cell_count, int64_t cells,
                      const int32_t *__restrict__ gate) {
    pdl_entry();
    if (gate && *gate == 0) return;  // gated rebuild: nothing to do
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int b = batch ? batch[n] : 0;
    const SysInfo s = info[b];
    int cx, cy, cz;
    point_cell(pos[3LL * n], pos[3LL * n + 1], pos[3LL * n + 2], s, cx, cy, cz);
    int64_t c = cell_off[b] + ((int64_t)cx * s.nc[1] + cy) * s.nc[2] + cz;
    if (c >= cells) c = cells - 1;  // unreachable when the budget holds
    cell_of[n] = (int32_t)c;
    atomicAdd(&cell_count[c], 1);
}

__global__ void k_scatter(const float *__restrict__ pos, int N, const int32_t *__restrict__ cell_of,
                          const int32_t *__restrict__ cell_start, int32_t *__restrict__ cell_fill,
                          int32_t *__restrict__ sorted, float4 *__restrict__ spos, const int32_t *__restrict__ gate) {
    pdl_entry();
    if (gate && *gate == 0) return;  // gated rebuild: nothing to do
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int c = cell_of[n];
    const int slot = cell_start[c] + atomicAdd(&cell_fill[c], 1);
    sorted[slot] = n;
    spos[slot] = make_float4(pos[3LL * n], pos[3LL * n + 1], pos[3LL * n + 2], __int_as_float(n));
}

// distinct neighbour cells of cell c along one axis (wrapping when periodic)
__device__ __forceinline__ int axis_neighbors(int c, int nc, int pbc, int out[3]) {
    if (nc <= 3) {
        for (int k = 0; k < nc; ++k) out[k] = k;
        return nc;
    }
    int m = 0;
    for (int o = -1; o <= 1; ++o) {
        int x = c + o;
        if (pbc) x = (x + nc) % nc;
        else if (x < 0 || x >= nc) continue;
        out[m++] = x;
    }
    return m;
}

// Visits every candidate j of atom i (same system, neighbouring cells) with
// one warp; `fn(j, ok)` is called by all lanes in lock-step, once per chunk of
// 32 candidates (lanes past the last candidate get j = -1, ok = false).
// Cells are numbered z-fastest, so the neighbouring cells along z of one
// (x, y) column form one run of consecutive cells (two when the run wraps
// around a periodic face), whose atoms are one contiguous range of the
// cell-sorted order.  Lane r first loads the bounds of range r (at most 27,
// 9 without wrap), a warp scan lays the ranges end to end, and the warp then
// walks the concatenated candidates 32 at a time, two chunks' loads in
// flight: each lane finds the range of its candidate by a five-step search
// over the scanned offsets (shuffles, the same steps in every lane).
template <class Fn>
__device__ __forceinline__ void for_candidates(int i, const float *__restrict__ pos,
                                               const int32_t *__restrict__ batch,
                                               const SysInfo *__restrict__ info,
                                               const int32_t *__restrict__ cell_off,
                                               const int32_t *__restrict__ cell_start,
                                               const float4 *__restrict__ spos, float rc2, Fn fn) {
    const int lane = threadIdx.x & 31;
    const int b = batch ? batch[i] : 0;
    const SysInfo s = info[b];
    const float xi = pos[3LL * i], yi = pos[3LL * i + 1], zi = pos[3LL * i + 2];
    int cx, cy, cz;
    point_cell(xi, yi, zi, s, cx, cy, cz);
    int nx[3], ny[3], nz[3];
    const int mx = axis_neighbors(cx, s.nc[0], s.pbc, nx);
    const int my = axis_neighbors(cy, s.nc[1], s.pbc, ny);
    const int mz = axis_neighbors(cz, s.nc[2], s.pbc, nz);
    // the z cells in ascending order, merged into runs of consecutive cells
    int z0 = nz[0], z1 = mz > 1 ? nz[1] : 0x7fffffff, z2 = mz > 2 ? nz[2] : 0x7fffffff, t;
    if (z0 > z1) { t = z0; z0 = z1; z1 = t; }
    if (z1 > z2) { t = z1; z1 = z2; z2 = t; }
    if (z0 > z1) { t = z0; z0 = z1; z1 = t; }
    int ra0 = z0, ra1 = z0, rb0 = 0, rb1 = -1, rc0 = 0, rc1 = -1, nrun = 1;
    auto extend = [&](int z) {  // append z (ascending) to the last run or open a new one
        if (nrun == 1) {
            if (z == ra1 + 1) ra1 = z;
            else { rb0 = rb1 = z; nrun = 2; }
        } else if (nrun == 2) {
            if (z == rb1 + 1) rb1 = z;
            else { rc0 = rc1 = z; nrun = 3; }
        }
    };
    if (mz > 1) extend(z1);
    if (mz > 2) extend(z2);
    const int R = mx * my * nrun;  // ranges, <= 27
    const int off = cell_off[b];
    int p0 = 0, len = 0;
    if (lane < R) {
        const int run = lane % nrun, rxy = lane / nrun;
        const int a = rxy / my, bb = rxy % my;
        const int xa = a == 0 ? nx[0] : (a == 1 ? nx[1] : nx[2]);
        const int yb = bb == 0 ? ny[0] : (bb == 1 ? ny[1] : ny[2]);
        const int lo = run == 0 ? ra0 : (run == 1 ? rb0 : rc0);
        const int hi = run == 0 ? ra1 : (run == 1 ? rb1 : rc1);
        const int col0 = off + (xa * s.nc[1] + yb) * s.nc[2];
        p0 = cell_start[col0 + lo];
        len = cell_start[col0 + hi + 1] - p0;
    }
    // exclusive offsets of the ranges laid end to end
    int incl = len;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += v;
    }
    const int excl = incl - len;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int c0 = 0; c0 < total; c0 += 64) {
        float4 q[2];
        bool has[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int tc = c0 + 32 * u + lane;
            has[u] = tc < total;
            if (c0 + 32 * u >= total) continue;  // the same in every lane
            // last range whose offset is <= tc (it holds tc when tc < total)
            int r = 0;
            if (R > 1) {  // the same in every lane
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int cand = r + step;
                    const int e = __shfl_sync(0xffffffffu, excl, cand & 31);
                    if (cand < R && e <= tc) r = cand;
                }
            }
            const int rp0 = __shfl_sync(0xffffffffu, p0, r);
            const int rex = __shfl_sync(0xffffffffu, excl, r);
            if (has[u]) q[u] = spos[rp0 + (tc - rex)];
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (c0 + 32 * u >= total) break;  // the same in every lane
            bool ok = false;
            int j = -1;
            if (has[u]) {
                j = __float_as_int(q[u].w);
                float dx = __fsub_rn(xi, q[u].x), dy = __fsub_rn(yi, q[u].y), dz = __fsub_rn(zi, q[u].z);
                mic(dx, dy, dz, s);
                const float d2 = norm2_rn(dx, dy, dz);
                ok = (j != i) && (d2 < rc2);
            }
            fn(j, ok);
        }
    }
}

__global__ void k_pair_count(const float *__restrict__ pos, const int32_t *__restrict__ batch, int N,
                             const SysInfo *__restrict__ info, const int32_t *__restrict__ cell_off,
                             const int32_t *__restrict__ cell_start, const float4 *__restrict__ spos,
                             float rc2, int32_t *__restrict__ rowcnt, const int32_t *__restrict__ gate) {
    pdl_entry();
    if (gate && *gate == 0) return;  // gated rebuild: nothing to do
    const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (i >= N) return;
    int cnt = 0;
    for_candidates(i, pos, batch, info, cell_off, cell_start, spos, rc2, [&](int j, bool ok) {
        cnt += __popc(__ballot_sync(0xffffffffu, ok));
    });
    if ((threadIdx.x & 31) == 0) rowcnt[i] = cnt;
}

// More pairs than the capacity: flag it (n_pairs keeps the required count)
// and clamp the row offsets to the capacity, so that the truncated list
// never sends a reader past the end of col.
__global__ void k_cap_check(const int64_t *__restrict__ n_pairs, int64_t cap, int32_t *__restrict__ row_ptr, int N,
                            int32_t *status, const int32_t *__restrict__ gate) {
    pdl_entry();
    if (gate && *gate == 0) return;  // gated rebuild: nothing to do
    if (*n_pairs <= cap) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) set_status(status, TNET_ERR_CAPACITY);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t <= N; t += (int64_t)gridDim.x * blockDim.x)
        if (row_ptr[t] > cap) row_ptr[t] = (int32_t)cap;
}

constexpr int kFillWarps = 4;

__global__ void __launch_bounds__(kFillWarps * 32)
k_pair_fill(const float *__restrict__ pos, const int32_t *__restrict__ batch, int N,
            const SysInfo *__restrict__ info, const int32_t *__restrict__ cell_off,
            const int32_t *__restrict__ cell_start, const float4 *__restrict__ spos, float rc2,
            const int32_t *__restrict__ row_ptr, int32_t *__restrict__ col, int64_t cap,
            const int32_t *__restrict__ gate) {
    pdl_entry();
    if (gate && *gate == 0) return;  // gated rebuild: nothing to do
    __shared__ int32_t buf[kFillWarps][kMaxRowSorted];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kFillWarps + w;
    if (i >= N) return;
    const int64_t r0 = row_ptr[i];
    const int rlen = row_ptr[i + 1] - row_ptr[i];
    int32_t *sb = buf[w];
    const bool in_smem = rlen <= kMaxRowSorted;
    int cnt = 0;
    // rlen is the count pass's result, clamped when the list overflowed the
    // capacity: write no more than that
    for_candidates(i, pos, batch, info, cell_off, cell_start, spos, rc2, [&](int j, bool ok) {
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        const int slot = cnt + __popc(m & ((1u << lane) - 1u));
        if (ok && slot < rlen) {
            if (in_smem) sb[slot] = j;
            else col[r0 + slot] = j;
        }
        cnt += __popc(m);
    });
    cnt = cnt < rlen ? cnt : rlen;
    __syncwarp();
    if (in_smem) {
        int P = 1;
        while (P < cnt) P <<= 1;
        for (int k = cnt + lane; k < P; k += 32) sb[k] = 0x7fffffff;
        __syncwarp();
        for (int k = 2; k <= P; k <<= 1) {
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int t = lane; t < P; t += 32) {
                    const int u = t ^ jj;
                    if (u > t) {
                        const int32_t a = sb[t], b = sb[u];
                        const bool up = (t & k) == 0;
                        if ((a > b) == up) {
                            sb[t] = b;
                            sb[u] = a;
                        }
                    }
                }
                __syncwarp();
            }
        }
        for (int k = lane; k < cnt; k += 32) col[r0 + k] = sb[k];
    } else if (lane == 0) {
        // pathological row: sort in place in global memory
        for (int a = 1; a < cnt; ++a) {
            const int32_t v = col[r0 + a];
            int b = a - 1;
            while (b >= 0 && col[r0 + b] > v) {
                col[r0 + b + 1] = col[r0 + b];
                --b;
            }
            col[r0 + b + 1] = v;
        }
    }
}

// Single candidate pass: one warp per atom collects its neighbours (one walk
// of the 27 cells), sorts them in shared memory and writes the sorted row to
// the atom's slot of the slab (kSlabWidth columns), with the row's count.  A
// row longer than kSlabWidth raises `over`; the two-pass fill then runs
// instead of the copy (gated on it), so the result never depends on the slab.
__global__ void __launch_bounds__(kFillWarps * 32)
k_pair_fill_slab(const float *__restrict__ pos, const int32_t *__restrict__ batch, int N,
                 const SysInfo *__restrict__ info, const int32_t *__restrict__ cell_off,
                 const int32_t *__restrict__ cell_start, const float4 *__restrict__ spos, float rc2,
                 int32_t *__restrict__ rowcnt, int32_t *__restrict__ slab, int32_t *__restrict__ over) {
    pdl_entry();
    __shared__ int32_t buf[kFillWarps][kSlabWidth];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kFillWarps + w;
    if (i >= N) return;
    int32_t *sb = buf[w];
    int cnt = 0;
    for_candidates(i, pos, batch, info, cell_off, cell_start, spos, rc2, [&](int j, bool ok) {
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        const int slot = cnt + __popc(m & ((1u << lane) - 1u));
        if (ok && slot < kSlabWidth) sb[slot] = j;
        cnt += __popc(m);
    });
    if (lane == 0) rowcnt[i] = cnt;
    if (cnt > kSlabWidth) {
        if (lane == 0) *over = 1;
        return;
    }
    __syncwarp();
    int P = 1;
    while (P < cnt) P <<= 1;
    for (int k = cnt + lane; k < P; k += 32) sb[k] = 0x7fffffff;
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int t = lane; t < P; t += 32) {
                const int u = t ^ jj;
                if (u > t) {
                    const int32_t a = sb[t], b = sb[u];
                    const bool up = (t & k) == 0;
                    if ((a > b) == up) {
                        sb[t] = b;
                        sb[u] = a;
                    }
                }
            }
            __syncwarp();
        }
    }
    int32_t *dst = slab + (int64_t)i * kSlabWidth;
    for (int k = lane; k < cnt; k += 32) dst[k] = sb[k];
}

// Rows of the slab into the CSR (warp per row), each within the row offsets
// (clamped to the capacity when the list overflowed).  Skipped when a row did
// not fit the slab: the gated two-pass fill writes the list then.
__global__ void k_slab_copy(const int32_t *__restrict__ slab, const int32_t *__restrict__ row_ptr, int N,
                            int32_t *__restrict__ col, const int32_t *__restrict__ over) {
    pdl_entry();
    if (*over) return;
    const int lane = threadIdx.x & 31;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < N;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int r0 = row_ptr[i], n = row_ptr[i + 1] - r0;
        const int32_t *src = slab + i * kSlabWidth;
        for (int k = lane; k < n; k += 32) col[r0 + k] = src[k];
    }
}

int neighbors_impl(tnet_ctx *ctx, int N, int S, const float *pos, const int32_t *batch,
                   const float *box, float cutoff, int32_t *row_ptr, int32_t *col, int64_t cap,
                   int64_t *n_pairs_dev, int32_t *status, cudaStream_t st, const int32_t *gate) {
    const Layout &L = ctx->lay;
    int32_t *sys_start = wsp<int32_t>(ctx, L.sys_start), *sys_end = wsp<int32_t>(ctx, L.sys_end);
    SysInfo *info = wsp<SysInfo>(ctx, L.sysinfo);
    int32_t *ncell = wsp<int32_t>(ctx, L.sys_ncell);
    int32_t *cell_count = wsp<int32_t>(ctx, L.cell_count), *cell_start = wsp<int32_t>(ctx, L.cell_start);
    int32_t *cell_fill = wsp<int32_t>(ctx, L.cell_fill), *cell_of = wsp<int32_t>(ctx, L.cell_of);
    int32_t *sorted = wsp<int32_t>(ctx, L.sorted), *rowcnt = wsp<int32_t>(ctx, L.rowcnt);
    int32_t *tmp = wsp<int32_t>(ctx, L.scan_tmp);
    float4 *spos = wsp<float4>(ctx, L.spos);
    const int cells = (int)L.cells;
    ProfSeq pf(ctx, st);
    pf.mark(P_NBR);

    auto zero = [&](int32_t *p, int64_t n) -> int {
        if (!gate) {
            TNET_CUDA_TRY(cudaMemsetAsync(p, 0, sizeof(int32_t) * n, st));
            return TNET_OK;
        }
        launch(k_zero_i32, (unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, st, p, n, gate);
        count_launch();
        return TNET_OK;
    };
    int zrc = zero(sys_start, S);
    if (!zrc) zrc = zero(sys_end, S);
    if (!zrc) zrc = zero(cell_count, cells + 1LL);
    if (!zrc) zrc = zero(cell_fill, cells);
    if (zrc) return zrc;
    if (N > 0) {
        launch(k_sys_bounds, (N + 255) / 256, 256, 0, st, batch, N, S, sys_start, sys_end, status, gate);
        count_launch();
        TNET_LAUNCH_CHECK();
    }
    launch(k_sys_setup, S, 256, 0, st, pos, box, cutoff, sys_start, sys_end, info, ncell, status, gate);
    count_launch();
    TNET_LAUNCH_CHECK();
    int rc = scan_exclusive_i32(ncell, ncell, S, tmp, nullptr, nullptr, st, gate);
    if (rc) return rc;
    if (N > 0) {
        launch(k_bin, (N + 255) / 256, 256, 0, st, pos, batch, N, info, ncell, cell_of, cell_count, cells, gate);
        count_launch();
        TNET_LAUNCH_CHECK();
    }
    rc = scan_exclusive_i32(cell_count, cell_start, cells, tmp, nullptr, nullptr, st, gate);
    if (rc) return rc;
    // one candidate pass into the row slab, unless the context has none or
    // the call is a gated rebuild (MD): then a count pass and a fill pass
    const bool one_pass = L.slab_width > 0 && !gate && N > 0;
    int32_t *over = one_pass ? wsp<int32_t>(ctx, L.slab_over) : nullptr;
    if (N > 0) {
        launch(k_scatter, (N + 255) / 256, 256, 0, st, pos, N, cell_of, cell_start, cell_fill, sorted, spos, gate);
        count_launch();
        TNET_LAUNCH_CHECK();
        if (one_pass) {
            TNET_CUDA_TRY(cudaMemsetAsync(over, 0, sizeof(int32_t), st));
            launch(k_pair_fill_slab, (N + kFillWarps - 1) / kFillWarps, kFillWarps * 32, 0, st, pos, batch, N, info,
                   ncell, cell_start, spos, cutoff * cutoff, rowcnt, wsp<int32_t>(ctx, L.slab), over);
        } else {
            launch(k_pair_count, (int)(((int64_t)N * 32 + 255) / 256), 256, 0, st, pos, batch, N, info, ncell,
                   cell_start, spos, cutoff * cutoff, rowcnt, gate);
        }
        count_launch();
        TNET_LAUNCH_CHECK();
    }
    rc = scan_exclusive_i32(rowcnt, row_ptr, N, tmp, nullptr, n_pairs_dev, st, gate);
    if (rc) return rc;
    launch(k_cap_check, (N + 256) / 256 < 1024 ? (N + 256) / 256 : 1024, 256, 0, st, n_pairs_dev, cap, row_ptr, N,
           status, gate);
    count_launch();
    TNET_LAUNCH_CHECK();
    if (N > 0) {
        if (one_pass) {
            const int nb = (int)(((int64_t)N * 32 + 255) / 256);
            launch(k_slab_copy, nb < 4096 ? nb : 4096, 256, 0, st, wsp<int32_t>(ctx, L.slab), row_ptr, N, col, over);
            count_launch();
            TNET_LAUNCH_CHECK();
        }
        // the fill pass; in one-pass mode gated on a row that did not fit
        launch(k_pair_fill, (N + kFillWarps - 1) / kFillWarps, kFillWarps * 32, 0, st, pos, batch, N, info, ncell,
               cell_start, spos, cutoff * cutoff, row_ptr, col, cap, one_pass ? over : gate);
        count_launch();
        TNET_LAUNCH_CHECK();
    }
    return TNET_OK;
}

}  // namespace tnet
