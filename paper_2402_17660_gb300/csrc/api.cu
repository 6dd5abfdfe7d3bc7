// C ABI entry points, context and workspace layout, and the MD step.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>

#include "internal.cuh"

namespace tnet {

int validate_desc(const tnet_model_desc *d) {
    if (!d) return TNET_ERR_ARG;
    if (d->F < 64 || d->F > 512 || d->F % 64) return TNET_ERR_ARG;
    if (d->K < 8 || d->K > 64 || d->K % 8) return TNET_ERR_ARG;
    if (d->L < 0 || d->L > 8) return TNET_ERR_ARG;
    if (d->max_z < 1 || d->max_z > 128) return TNET_ERR_ARG;
    if (!(d->cutoff_upper > d->cutoff_lower) || d->cutoff_lower < 0.f) return TNET_ERR_ARG;
    if (d->precision < 0 || d->precision > 2) return TNET_ERR_ARG;
    if (d->recompute_edges < 0 || d->recompute_edges > 1) return TNET_ERR_ARG;
    if (d->radial_table != 0 && (d->radial_table < 256 || d->radial_table > 16384)) return TNET_ERR_ARG;
    return TNET_OK;
}

int build_layout(const tnet_model_desc *d, int N, int S, int64_t E, Layout *L) {
    if (validate_desc(d) || N < 1 || S < 1 || E < 0) return TNET_ERR_ARG;
    size_t off = 0;
    auto take = [&](int64_t bytes) {
        const size_t o = off;
        off += ((size_t)(bytes > 0 ? bytes : 0) + 255) & ~(size_t)255;
        return o;
    };
    const int64_t F = d->F, K = d->K, NL = d->L, Z = d->max_z;
    const int64_t n9 = 9LL * N * F;
    const int64_t cells = 2LL * N + 8LL * S + 64;
    const int64_t U = E / 2 + 1;
    const int64_t f = 4, i = 4;
    L->node9 = n9;
    L->cells = cells;
    L->maxU = U;
    int64_t big = N + 1;
    if (cells + 1 > big) big = cells + 1;
    if (S + 1 > big) big = S + 1;
    // neighbor search
    L->sys_start = take(i * S);
    L->sys_end = take(i * S);
    L->sysinfo = take(sizeof(SysInfo) * S);
    L->sys_ncell = take(i * (S + 1));
    L->cell_count = take(i * (cells + 1));
    L->cell_start = take(i * (cells + 1));
    L->cell_fill = take(i * cells);
    L->cell_of = take(i * N);
    L->sorted = take(i * N);
    L->spos = take(16LL * N);
    L->rowcnt = take(i * (N + 1));
    L->scan_tmp = take(i * (big / 4096 + 16));
    // graph prep
    L->rp_safe = take(i * (N + 1));
    L->rev = take(i * E);
    L->pair_of = take(i * E);
    L->uedge = take(8 * U);
    L->ucnt = take(i * (N + 1));
    L->nu = take(i * 4);
    // node buffers
    L->Ta = take(f * Z * F);
    L->Tb = take(f * Z * F);
    L->Xraw = take(f * n9);
    L->Uemb = take(f * n9);
    L->n0 = take(f * N * F);
    L->as1 = take(f * N * 2 * F);
    L->hs1 = take(f * N * 2 * F);
    L->as2 = take(f * N * 3 * F);
    L->s = take(f * N * 3 * F);
    L->ln0 = take(8LL * N);
    L->Xin = take(f * n9 * (NL > 0 ? NL : 1));
    L->qn = take(f * N * F * NL);
    L->Xn = take(f * n9 * NL);
    L->Y = take(f * n9 * NL);
    L->M = take(f * n9 * NL);
    L->Tn = take(f * n9 * NL);
    L->dX = take(f * n9 * NL);
    L->Xfin = take(f * n9);
    L->h = take(f * N * 3 * F);
    L->hn = take(f * N * 3 * F);
    L->lno = take(8LL * N);
    L->ao = take(f * N * F);
    L->o = take(f * N * F);
    L->at = take(f * N * F / 2);
    L->t = take(f * N * F / 2);
    L->Ei = take(f * N);
    // edge MLP (none of it in table mode: the consumers evaluate the tables)
    const int64_t nt = d->radial_table;
    const int64_t rm = nt > 0 ? 0 : 1;  // the per-pair radial MLP runs
    L->eu = take(f * U * K * rm);
    L->phiu = take(f * U);
    L->geo = take(16 * U);
    // (one set per layer, which the reverse pass reads, unless it recomputes
    // them; none in table mode, where the message kernels evaluate the tables)
    const int64_t NLm = (NL > 0 && !d->recompute_edges) ? NL : 1;
    L->a1 = take(f * U * F * NLm * rm);
    L->h1 = take(f * U * F * NLm * rm);
    L->a2 = take(f * U * 2 * F * NLm * rm);
    L->h2 = take(f * U * 2 * F * NLm * rm);
    L->a3 = take(f * U * 3 * F * NLm * rm);
    // (no per-pair filter g = phi SiLU(a3): the message kernels form it from a3)
    // reverse pass
    L->gXa = take(f * n9);
    L->gXb = take(f * n9);
    L->gdX = take(f * n9);
    L->gTn = take(f * n9);
    L->gM = take(f * n9);
    L->gY = take(f * n9);
    L->gat = take(f * N * F / 2);
    L->gao = take(f * N * F);
    L->ghn = take(f * N * 3 * F);
    L->gh = take(f * N * 3 * F);
    L->gU = take(f * n9);
    L->gas2 = take(f * N * 3 * F);
    L->gas1 = take(f * N * 2 * F);
    L->gn0 = take(f * N * F);
    L->gq0 = take(f * N * F);
    L->gg = take(f * U * 3 * F * rm);
    L->ga2 = take(f * U * 2 * F * rm);
    L->ga1 = take(f * U * F * rm);
    L->ge = take(f * U * K * rm);
    L->gphiu = take(f * U);
    L->gvec = take(f * 3 * E);
    L->fu = take(f * U * 3 * F * rm);
    L->gfu = take(f * U * 3 * F * rm);
    L->ue = take(i * U);
    L->edge_g = take(16 * E);
    L->gp = take(f * 3 * U);
    L->q0 = take(f * N * F);
    L->gEi = take(f * N);
    L->gA_atom = take(f * N * F);
    L->gB_atom = take(f * N * F);
    L->zsplits = 32;
    L->zpart = take(f * 2 * L->zsplits * Z * F);
    L->wpart_floats = 4LL << 20;
    L->wpart = take(f * L->wpart_floats);
    L->w3p = take(f * (NL > 0 ? NL : 1) * (6LL * F * F + 3 * F));
    // tabulated radial functions (radial_table = n > 0): Hermite coefficients
    // [n-1][3F] float4 of the projections f and of each layer's filter g, the
    // FP64 scratch of their construction and the per-pair distance
    L->tab = take(f * (nt > 0 ? (NL + 1) * (nt - 1) * 4 * 3 * F : 0));
    L->tab_tmp = take(8 * (nt > 0 ? nt * (2 * K + 2 + 12 * F) : 0));
    L->dist = take(f * (nt > 0 ? U : 0));
    // tensor-core modes: weight operands (bf16 forward + transposed copies,
    // or fp32 TF32 residuals + transposed high parts; the 3xTF32 GEMMs of the
    // BF16 mode use the latter), and in BF16 mode the bf16 copies of the node
    // tensor and radial-MLP activations the BF16 GEMMs read (3xTF32 reads the
    // fp32 activations themselves)
    const int prec = d->precision;
    const int64_t esz = prec == 1 ? 2 : 0;
    int64_t nw = 0;
    {
        nw += Z * F + F * 2 * F + F + 3 * F * K + 3 * F + 2 * F + 2 * F * F + 2 * F + 3 * F * 2 * F + 3 * F +
              3 * F * F;
        nw += NL * (F * K + F + 2 * F * F + 2 * F + 3 * F * 2 * F + 3 * F + 6 * F * F);
        nw += 6 * F + F * 3 * F + F + F / 2 * F + F / 2 + F / 2 + 1;
    }
    L->wbf_bytes = prec ? 3 * nw * 4 + 128 * 256 : 0;
    L->wbf = take(L->wbf_bytes);
    L->nbf = take(esz * n9);
    L->eu_bf = 0;
    L->h1_bf = take(esz * U * F * NLm * rm);
    L->h2_bf = take(esz * U * 2 * F * NLm * rm);
    L->ga3_bf = take(esz * U * 3 * F * rm);
    L->ga2_bf = take(esz * U * 2 * F * rm);
    L->ga1_bf = 0;
    L->gfu_bf = 0;
    // MD
    L->md_row_ptr = take(i * (N + 1));
    L->md_col = take(i * E);
    L->md_npairs = take(8);
    L->md_forces = take(f * 3 * N);
    L->md_energy = take(8);
    L->md_pos_ref = take(f * 3 * N);
    L->md_step = take(i * 4);
    L->md_need = take(i * 4);
    L->md_rebuilds = take(8);
    // the single-pass neighbor search's row slab (last, so that the neighbor
    // part at the front of the layout keeps its size)
    L->slab_width = kSlabWidth;
    L->slab = take(i * (int64_t)N * kSlabWidth);
    L->slab_over = take(i * 4);
    L->total = off;
    return TNET_OK;
}

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

ProfSeq::ProfSeq(tnet_ctx *ctx, cudaStream_t s) : c(ctx), st(s), slot(-1), active(false) {
    if (!c || !c->prof_on) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    active = true;
}
void ProfSeq::mark(int tag) {
    if (!active) return;
    if (slot >= 0) {
        cudaEventRecord(c->prof_ev[2 * slot + 1], st);
        slot = -1;
    }
    if (tag >= 0 && c->prof_n < c->prof_cap) {
        slot = c->prof_n++;
        c->prof_tag[slot] = tag;
        cudaEventRecord(c->prof_ev[2 * slot], st);
    }
}

}  // namespace tnet

using namespace tnet;

thread_local int tnet::tl_pdl = 1;

// Candidate values of each tuning knob (TuneKnob) and the default's index.
static const int kTuneCandidates[T_NKNOBS][4] = {{1, 2, 3, 4}, {192, 128, 0, 0}, {256, 128, 0, 0}, {4, 8, 16, 0},
                                                 {4, 8, 16, 0}, {1, 0, 0, 0}, {0, 1, 4, 3}, {2, 1, 4, 0}};
static const int kTuneCount[T_NKNOBS] = {4, 2, 2, 3, 3, 2, 4, 3};
// Defaults: the shapes the autotuner picks on most measured workloads (24k to
// 96k atoms, both tensor-core precisions).  Programmatic launch is on only for
// contexts of at most kPdlMaxAtoms atoms, the launch-bound systems it speeds up;
// from a few thousand atoms on it was measured to slow the step by 5-15%.
static const int kTuneDefault[T_NKNOBS] = {2, 0, 0, 2, 2, 1, 3, 0};
static const int64_t kPdlMaxAtoms = 1024;
static const char *kTuneNames[T_NKNOBS] = {"gemm_ctas_per_sm",   "tc_tile_n_3f",        "tc_tile_n_2f",
                                           "row_blocks_per_sm",  "pair_blocks_per_sm",  "programmatic_launch",
                                           "message_kernel",     "tc_cluster"};

static const char *kTagNames[P_NTAGS] = {
    "neighbors", "graph_prep", "emb_edges", "emb_node", "mlp1", "mlp2", "mlp3", "message",
    "node_mix", "node_elem", "output", "output_bwd", "node_bwd", "message_bwd", "mlp_elem_bwd",
    "mlp3_bwd", "mlp2_bwd", "mlp1_bwd", "emb_node_bwd", "emb_edges_bwd", "forces"};

extern "C" {

const char *tnet_status_string(int s) {
    switch (s) {
        case TNET_OK: return "ok";
        case TNET_ERR_ARG: return "invalid argument";
        case TNET_ERR_CAPACITY: return "pair capacity exceeded";
        case TNET_ERR_BOX: return "box not lower-triangular or narrower than twice the cutoff";
        case TNET_ERR_NAN: return "non-finite position";
        case TNET_ERR_CUDA: return "CUDA runtime error";
        case TNET_ERR_TIMEOUT: return "device wait timed out";
        case TNET_ERR_WORKSPACE: return "workspace too small or misaligned";
        case TNET_ERR_Z: return "atomic number out of range";
        case TNET_ERR_UNSUPPORTED: return "not supported by this build";
        case TNET_ERR_SKIN: return "reserved (skin violations trigger a rebuild)";
        default: return "unknown status";
    }
}

int64_t tnet_weights_count(const tnet_model_desc *d) {
    if (validate_desc(d)) return -1;
    return weight_offsets(d, nullptr, nullptr);
}

int64_t tnet_workspace_bytes(const tnet_model_desc *d, int max_atoms, int max_systems, int64_t max_pairs) {
    Layout L;
    if (build_layout(d, max_atoms, max_systems, max_pairs, &L)) return -1;
    return (int64_t)L.total;
}

int tnet_create(tnet_ctx **out, const tnet_model_desc *d, int max_atoms, int max_systems,
                int64_t max_pairs, void *workspace, size_t workspace_bytes) {
    if (!out) return TNET_ERR_ARG;
    *out = nullptr;
    Layout L;
    int rc = build_layout(d, max_atoms, max_systems, max_pairs, &L);
    if (rc) return rc;
    if (max_pairs > 0x7fffffffLL || max_atoms > (1 << 28)) return TNET_ERR_ARG;
    if (!workspace || ((uintptr_t)workspace & 255) || workspace_bytes < L.total) return TNET_ERR_WORKSPACE;
    tnet_ctx *c = (tnet_ctx *)calloc(1, sizeof(tnet_ctx));
    if (!c) return TNET_ERR_ARG;
    c->d = *d;
    c->max_atoms = max_atoms;
    c->max_systems = max_systems;
    c->max_pairs = max_pairs;
    c->ws = (char *)workspace;
    c->ws_bytes = workspace_bytes;
    c->lay = L;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        free(c);
        return TNET_ERR_CUDA;
    }
    RadialParams &rp = c->rp;
    rp.rc = d->cutoff_upper;
    rp.rl = d->cutoff_lower;
    rp.K = d->K;
    const double start = exp(-(double)(d->cutoff_upper - d->cutoff_lower));
    rp.alpha = (float)(5.0 / (double)(d->cutoff_upper - d->cutoff_lower));
    rp.beta = (float)pow((2.0 / d->K) * (1.0 - start), -2.0);
    rp.mu0 = (float)start;
    rp.dmu = (float)((1.0 - start) / (d->K - 1));
    for (int k = 0; k < T_NKNOBS; ++k) c->tune[k] = kTuneCandidates[k][kTuneDefault[k]];
    if (max_atoms <= kPdlMaxAtoms) c->tune[T_PDL] = 1;
    rc = tnet_kernel_setup(c);
    if (rc) {
        free(c);
        return rc;
    }
    *out = c;
    return TNET_OK;
}

int tnet_destroy(tnet_ctx *c) {
    if (!c) return TNET_ERR_ARG;
    if (c->md_exec) cudaGraphExecDestroy(c->md_exec);
    if (c->prof_ev) {
        for (int k = 0; k < 2 * c->prof_cap; ++k) cudaEventDestroy(c->prof_ev[k]);
        free(c->prof_ev);
        free(c->prof_tag);
    }
    free(c);
    return TNET_OK;
}

int64_t tnet_launch_count(void) { return g_launches.load(); }

int tnet_tuning_knobs(void) { return T_NKNOBS; }
const char *tnet_tuning_name(int knob) { return (knob >= 0 && knob < T_NKNOBS) ? kTuneNames[knob] : nullptr; }
int tnet_tuning_candidates(int knob, int32_t *values, int max) {
    if (knob < 0 || knob >= T_NKNOBS || !values) return -1;
    const int n = kTuneCount[knob] < max ? kTuneCount[knob] : max;
    for (int i = 0; i < n; ++i) values[i] = kTuneCandidates[knob][i];
    return kTuneCount[knob];
}
int tnet_get_tuning(tnet_ctx *c, int32_t *knobs, int n) {
    if (!c || !knobs || n < 0) return TNET_ERR_ARG;
    for (int k = 0; k < n && k < T_NKNOBS; ++k) knobs[k] = c->tune[k];
    return TNET_OK;
}
int tnet_set_tuning(tnet_ctx *c, const int32_t *knobs, int n) {
    if (!c || !knobs || n < 0 || n > T_NKNOBS) return TNET_ERR_ARG;
    for (int k = 0; k < n; ++k) {
        bool ok = false;
        for (int i = 0; i < kTuneCount[k]; ++i) ok |= kTuneCandidates[k][i] == knobs[k];
        if (!ok) return TNET_ERR_ARG;
    }
    for (int k = 0; k < n; ++k) c->tune[k] = knobs[k];
    return TNET_OK;
}

const char *tnet_profile_tag(int tag) { return (tag >= 0 && tag < P_NTAGS) ? kTagNames[tag] : nullptr; }

int tnet_profile(tnet_ctx *c, int enable) {
    if (!c) return TNET_ERR_ARG;
    if (enable && !c->prof_ev) {
        const int cap = 4096;
        c->prof_ev = (cudaEvent_t *)calloc(2 * cap, sizeof(cudaEvent_t));
        c->prof_tag = (int *)calloc(cap, sizeof(int));
        if (!c->prof_ev || !c->prof_tag) return TNET_ERR_ARG;
        for (int k = 0; k < 2 * cap; ++k) TNET_CUDA_TRY(cudaEventCreate(&c->prof_ev[k]));
        c->prof_cap = cap;
    }
    c->prof_on = enable ? 1 : 0;
    c->prof_n = 0;
    return TNET_OK;
}

int tnet_profile_read(tnet_ctx *c, int ntags, float *ms, int64_t *count) {
    if (!c || ntags < 0 || !ms || !count) return TNET_ERR_ARG;
    for (int t = 0; t < ntags; ++t) {
        ms[t] = 0.f;
        count[t] = 0;
    }
    for (int k = 0; k < c->prof_n; ++k) {
        TNET_CUDA_TRY(cudaEventSynchronize(c->prof_ev[2 * k + 1]));
        float e = 0.f;
        TNET_CUDA_TRY(cudaEventElapsedTime(&e, c->prof_ev[2 * k], c->prof_ev[2 * k + 1]));
        const int t = c->prof_tag[k];
        if (t < ntags) {
            ms[t] += e;
            count[t] += 1;
        }
    }
    return TNET_OK;
}

static int check_common(tnet_ctx *c, int N, int S, const float *pos, int32_t *status) {
    if (!c || !pos || !status) return TNET_ERR_ARG;
    if (N < 1 || N > c->max_atoms || S < 1 || S > c->max_systems) return TNET_ERR_ARG;
    return TNET_OK;
}

int tnet_neighbors(tnet_ctx *c, int N, int S, const float *pos, const int32_t *batch, const float *box,
                   float cutoff, int32_t *row_ptr, int32_t *col, int64_t cap, int64_t *n_pairs_dev,
                   int32_t *status, tnet_stream_t stream) {
    int rc = check_common(c, N, S, pos, status);
    if (rc) return rc;
    if (!row_ptr || !n_pairs_dev || (cap > 0 && !col)) return TNET_ERR_ARG;
    if (cap < 0 || cap > c->max_pairs || !(cutoff > 0.f) || !isfinite(cutoff)) return TNET_ERR_ARG;
    if (S > 1 && !batch) return TNET_ERR_ARG;
    PdlScope pdl_scope(c->tune[T_PDL]);
    return neighbors_impl(c, N, S, pos, batch, box, cutoff, row_ptr, col, cap, n_pairs_dev, status,
                          (cudaStream_t)stream);
}

int tnet_energy_forces(tnet_ctx *c, const float *w, int N, int S, const int32_t *z, const float *pos,
                       const int32_t *batch, const float *box, const int32_t *row_ptr,
                       const int32_t *col, const float *seed, double *energy, float *forces,
                       float *grad_w, int32_t *status, tnet_stream_t stream) {
    int rc = check_common(c, N, S, pos, status);
    if (rc) return rc;
    if (!w || !z || !row_ptr || !col || !energy) return TNET_ERR_ARG;
    if (S > 1 && !batch) return TNET_ERR_ARG;
    PdlScope pdl_scope(c->tune[T_PDL]);
    return energy_forces_impl(c, w, N, S, z, pos, batch, box, row_ptr, col, seed, energy, forces, grad_w,
                              status, (cudaStream_t)stream);
}

int tnet_radial_tables(tnet_ctx *c, const float *w, tnet_stream_t stream) {
    if (!c || !w || c->d.radial_table <= 0) return TNET_ERR_ARG;
    PdlScope pdl_scope(c->tune[T_PDL]);
    return radial_tables_impl(c, w, (cudaStream_t)stream);
}

int tnet_md_step(tnet_ctx *c, const float *w, int N, const int32_t *z, const float *inv_mass, float *pos,
                 float *vel, const float *box, float dt, float skin, int rebuild_every, int n_steps,
                 double *e_kin, double *e_pot, int32_t *status, tnet_stream_t stream) {
    int rc = check_common(c, N, 1, pos, status);
    if (rc) return rc;
    if (!w || !z || !inv_mass || !vel || (n_steps > 0 && (!e_kin || !e_pot))) return TNET_ERR_ARG;
    if (!(dt > 0.f) || !(skin >= 0.f) || rebuild_every < 1 || n_steps < 0) return TNET_ERR_ARG;
    PdlScope pdl_scope(c->tune[T_PDL]);
    return md_impl(c, w, N, z, inv_mass, pos, vel, box, dt, skin, rebuild_every, n_steps, e_kin, e_pot,
                   status, (cudaStream_t)stream);
}

int tnet_md_neighbor_list(tnet_ctx *c, int N, int32_t *row_ptr, int32_t *col, int64_t cap, int64_t *n_pairs,
                          tnet_stream_t stream) {
    if (!c || !row_ptr || !n_pairs || N < 1 || N > c->max_atoms || cap < 0 || (cap > 0 && !col)) return TNET_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const Layout &L = c->lay;
    TNET_CUDA_TRY(cudaMemcpyAsync(row_ptr, wsp<int32_t>(c, L.md_row_ptr), sizeof(int32_t) * (N + 1),
                                  cudaMemcpyDeviceToDevice, st));
    TNET_CUDA_TRY(cudaMemcpyAsync(n_pairs, wsp<int64_t>(c, L.md_npairs), sizeof(int64_t), cudaMemcpyDeviceToDevice,
                                  st));
    const int64_t n = cap < c->max_pairs ? cap : c->max_pairs;
    if (n > 0)
        TNET_CUDA_TRY(cudaMemcpyAsync(col, wsp<int32_t>(c, L.md_col), sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st));
    return TNET_OK;
}

int tnet_md_rebuilds(tnet_ctx *c, int64_t *count) {
    if (!c || !count) return TNET_ERR_ARG;
    TNET_CUDA_TRY(cudaMemcpy(count, wsp<int64_t>(c, c->lay.md_rebuilds), sizeof(int64_t), cudaMemcpyDeviceToHost));
    return TNET_OK;
}

}  // extern "C"
