// Velocity-Verlet molecular dynamics on top of the neighbor search and the
// energy/force pass.  One MD step is one energy evaluation plus one force
// backward pass (the paper's MD usage, Sec. 3 "Molecular Simulations").
// Blocks of `rebuild_every` steps are captured once into a CUDA graph (the
// paper's "Graph" optimisation, Sec. 2.5) and replayed; the only host work
// per block is one graph launch.
#include <string.h>

#include "internal.cuh"

namespace tnet {

constexpr float kAccel = 9.64853321e-3f;  // 1 eV / (A amu) in A / fs^2

__global__ void k_half_kick(float *__restrict__ vel, const float *__restrict__ F,
                            const float *__restrict__ inv_m, int N, float hdt) {
    pdl_entry();
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= 3LL * N) return;
    vel[t] += hdt * kAccel * F[t] * inv_m[t / 3];
}

// x += dt v; raise the rebuild flag when an atom is more than skin/2 from
// where it was at the last rebuild (two atoms closing in from outside
// cutoff + skin could then be within the cutoff)
__global__ void k_drift(float *__restrict__ pos, const float *__restrict__ vel, int N, float dt,
                        const float *__restrict__ ref, const float *__restrict__ box, float lim2,
                        int32_t *__restrict__ need) {
    pdl_entry();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float x = pos[3LL * i + k] + dt * vel[3LL * i + k];
        pos[3LL * i + k] = x;
        d[k] = x - ref[3LL * i + k];
    }
    if (box) mic_box(d[0], d[1], d[2], box);
    if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] > lim2) *need = 1;
}

__global__ void k_copy(float *__restrict__ dst, const float *__restrict__ src, int64_t n,
                       const int32_t *__restrict__ gate) {
    pdl_entry();
    if (gate && *gate == 0) return;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) dst[t] = src[t];
}

// after a rebuild slot: count it (periodic, or triggered by the flag) and
// clear the flag
__global__ void k_rebuild_done(int32_t *__restrict__ need, int64_t *__restrict__ count, int periodic) {
    pdl_entry();
    if (periodic || *need) ++*count;
    *need = 0;
}

// single block: kinetic energy (FP64, eV) and the step's records
__global__ void k_record(const float *__restrict__ vel, const float *__restrict__ inv_m, int N,
                         const double *__restrict__ epot_src, double *__restrict__ e_kin,
                         double *__restrict__ e_pot, int32_t *__restrict__ step) {
    pdl_entry();
    __shared__ double sm[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double vx = vel[3LL * i], vy = vel[3LL * i + 1], vz = vel[3LL * i + 2];
        acc += 0.5 * (vx * vx + vy * vy + vz * vz) / (double)inv_m[i];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
        const int s = *step;
        e_kin[s] = t / (double)kAccel;
        e_pot[s] = *epot_src;
        *step = s + 1;
    }
}

namespace {
struct MdArgs {
    const float *w;
    int N;
    const int32_t *z;
    const float *inv_m;
    float *pos, *vel;
    const float *box;
    float dt, skin;
    double *e_kin, *e_pot;
    int32_t *status;
};

// Neighbor list at cutoff + skin and the reference positions.  periodic:
// always; otherwise only if the drift raised the rebuild flag (the kernels
// are enqueued either way, so one graph serves every step, and return at
// once when the flag is clear).
int enqueue_rebuild(tnet_ctx *c, const MdArgs &a, bool periodic, cudaStream_t st) {
    const Layout &L = c->lay;
    const float rcut = c->d.cutoff_upper + a.skin;
    int32_t *need = wsp<int32_t>(c, L.md_need);
    const int32_t *gate = periodic ? nullptr : need;
    int rc = neighbors_impl(c, a.N, 1, a.pos, nullptr, a.box, rcut, wsp<int32_t>(c, L.md_row_ptr),
                            wsp<int32_t>(c, L.md_col), c->max_pairs, wsp<int64_t>(c, L.md_npairs), a.status,
                            st, gate);
    if (rc) return rc;
    launch(k_copy, (3 * a.N + 255) / 256, 256, 0, st, wsp<float>(c, L.md_pos_ref), a.pos, 3LL * a.N, gate);
    count_launch();
    launch(k_rebuild_done, 1, 1, 0, st, need, wsp<int64_t>(c, L.md_rebuilds), periodic ? 1 : 0);
    count_launch();
    TNET_LAUNCH_CHECK();
    return TNET_OK;
}

int enqueue_forces(tnet_ctx *c, const MdArgs &a, cudaStream_t st) {
    const Layout &L = c->lay;
    return energy_forces_impl(c, a.w, a.N, 1, a.z, a.pos, nullptr, a.box, wsp<int32_t>(c, L.md_row_ptr),
                              wsp<int32_t>(c, L.md_col), nullptr, wsp<double>(c, L.md_energy),
                              wsp<float>(c, L.md_forces), nullptr, a.status, st);
}

int enqueue_step(tnet_ctx *c, const MdArgs &a, bool rebuild, cudaStream_t st) {
    const Layout &L = c->lay;
    float *F = wsp<float>(c, L.md_forces);
    const int nb3 = (3 * a.N + 255) / 256, nb = (a.N + 255) / 256;
    launch(k_half_kick, nb3, 256, 0, st, a.vel, F, a.inv_m, a.N, 0.5f * a.dt);
    count_launch();
    const float lim = 0.5f * a.skin;
    launch(k_drift, nb, 256, 0, st, a.pos, a.vel, a.N, a.dt, wsp<float>(c, L.md_pos_ref), a.box, lim * lim,
                                wsp<int32_t>(c, L.md_need));
    count_launch();
    TNET_LAUNCH_CHECK();
    {
        int rc = enqueue_rebuild(c, a, rebuild, st);
        if (rc) return rc;
    }
    int rc = enqueue_forces(c, a, st);
    if (rc) return rc;
    launch(k_half_kick, nb3, 256, 0, st, a.vel, F, a.inv_m, a.N, 0.5f * a.dt);
    count_launch();
    launch(k_record, 1, 1024, 0, st, a.vel, a.inv_m, a.N, wsp<double>(c, L.md_energy), a.e_kin, a.e_pot,
                                 wsp<int32_t>(c, L.md_step));
    count_launch();
    TNET_LAUNCH_CHECK();
    return TNET_OK;
}
}  // namespace

int md_impl(tnet_ctx *c, const float *w, int N, const int32_t *z, const float *inv_m, float *pos,
            float *vel, const float *box, float dt, float skin, int R, int n_steps, double *e_kin,
            double *e_pot, int32_t *status, cudaStream_t st) {
    const MdArgs a{w, N, z, inv_m, pos, vel, box, dt, skin, e_kin, e_pot, status};
    TNET_CUDA_TRY(cudaMemsetAsync(wsp<int32_t>(c, c->lay.md_step), 0, sizeof(int32_t), st));
    TNET_CUDA_TRY(cudaMemsetAsync(wsp<int32_t>(c, c->lay.md_need), 0, sizeof(int32_t), st));
    TNET_CUDA_TRY(cudaMemsetAsync(wsp<int64_t>(c, c->lay.md_rebuilds), 0, sizeof(int64_t), st));
    // forces at the starting positions
    int rc = enqueue_rebuild(c, a, true, st);
    if (rc) return rc;
    rc = enqueue_forces(c, a, st);
    if (rc) return rc;
    const int full = n_steps / R, rem = n_steps % R;
    if (full > 0) {
        const void *key[8] = {w, z, inv_m, pos, vel, box, e_kin, e_pot};
        const int64_t keyi[6] = {N, R, (int64_t)(intptr_t)status, 0, 0, 0};
        const float keyf[3] = {dt, skin, 0.f};
        const bool same = c->md_exec && !memcmp(key, c->md_key, sizeof key) &&
                          !memcmp(keyi, c->md_keyi, sizeof keyi) && !memcmp(keyf, c->md_keyf, sizeof keyf);
        if (!same) {
            if (c->md_exec) {
                cudaGraphExecDestroy(c->md_exec);
                c->md_exec = nullptr;
            }
            cudaStream_t cs;
            TNET_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            TNET_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            int erc = TNET_OK;
            for (int k = 0; k < R && !erc; ++k) erc = enqueue_step(c, a, k == 0, cs);
            cudaError_t ce = cudaStreamEndCapture(cs, &g);
            cudaStreamDestroy(cs);
            if (erc) {
                if (g) cudaGraphDestroy(g);
                return erc;
            }
            if (ce != cudaSuccess) {
                fprintf(stderr, "libtnet: graph capture failed: %s\n", cudaGetErrorString(ce));
                return TNET_ERR_CUDA;
            }
            cudaGraphExec_t ex;
            ce = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) {
                fprintf(stderr, "libtnet: graph instantiate failed: %s\n", cudaGetErrorString(ce));
                return TNET_ERR_CUDA;
            }
            c->md_exec = ex;
            memcpy(c->md_key, key, sizeof key);
            memcpy(c->md_keyi, keyi, sizeof keyi);
            memcpy(c->md_keyf, keyf, sizeof keyf);
        }
        for (int b = 0; b < full; ++b) TNET_CUDA_TRY(cudaGraphLaunch(c->md_exec, st));
    }
    for (int k = 0; k < rem; ++k) {
        rc = enqueue_step(c, a, k == 0, st);
        if (rc) return rc;
    }
    return TNET_OK;
}

}  // namespace tnet
