/*
 * tnet.h - C ABI of libtnet: TensorNet energy and forces on one GB300 (sm_103a).
 *
 * The library computes what TorchMD-Net 2.0 (arXiv 2402.17660) describes as a
 * neural network potential: atomic positions R and embedding indices Z go in,
 * a per-sample scalar (the potential energy) and its negative gradient with
 * respect to the positions (the atomic forces) come out (Sec. 2, Background;
 * Fig. 1).  The representation model is TensorNet (Sec. 2.1.1), an
 * O(3)-equivariant message passing network on rank-2 Cartesian tensors, with
 * the hyperparameters of the paper's training example (Sec. 2.4, Table S4).
 * The graph comes from a periodic cell-list neighbor search (Sec. 2.5.1).
 *
 * Conventions shared by every entry point
 *   - Every pointer argument is a DEVICE pointer unless its comment says HOST.
 *     The caller owns all memory (inputs, outputs and the workspace handed to
 *     tnet_create); the library never allocates device memory.
 *   - Calls are ordered on the given CUDA stream and return as soon as the
 *     work is enqueued; they do not synchronise the host.  They issue no
 *     host<->device copies, so tnet_neighbors and tnet_energy_forces can be
 *     captured into a CUDA graph.
 *   - The int return value reports synchronous argument errors only (a
 *     tnet_status code).  Errors found on the device (pair capacity
 *     exceeded, box too small, bad atomic number, non-finite positions) are
 *     written to *status_dev (int32, device) with the first error winning;
 *     the caller zeroes it before the call, synchronises and reads it after.
 *   - Units: positions and box in Angstrom, energies in the model's unit
 *     (treated as eV by tnet_md_step), time in fs, mass in amu.
 *   - Arrays are C-contiguous; pos is [N][3] float32 (x, y, z per atom).
 *   - A context is not thread-safe: calls that share a context must be
 *     ordered on one stream.
 */
#ifndef TNET_H
#define TNET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL means the legacy default stream. */
typedef struct CUstream_st *tnet_stream_t;

typedef struct tnet_ctx tnet_ctx;

/* Model shape.  F: embedding dimension (channels), K: number of expnorm
 * radial basis functions, L: number of interaction layers, max_z: rows of
 * the atomic-number embedding table, cutoff_upper/lower: the cosine cutoff
 * interval in Angstrom (Sec. 2.4: embedding_dimension 128, num_layers 2,
 * num_rbf 32, max_z 100, cutoff 0..5 A).  precision: 0 = FP32 everywhere
 * (SIMT GEMMs); 1 = BF16 tensor-core GEMMs with FP32 accumulation for the
 * 2F/3F-wide radial-MLP layers and the I/A/S channel mixing; 2 = the same
 * GEMMs on the tensor cores in 3xTF32 (FP32 operands split into TF32 high
 * and residual parts), FP32-level accuracy.  Geometry, radial basis, the
 * num_rbf-wide layers and scatter-adds stay FP32 and the per-system energy
 * is reduced in FP64 in every mode.
 * Limits: F a multiple of 64 in [64, 512], K a multiple of 8 in [8, 64],
 * (precision 1 and 2 need F <= 256),
 * 0 <= L <= 8, 1 <= max_z <= 128, 0 <= cutoff_lower < cutoff_upper.
 * recompute_edges: 0 = the forward pass keeps every layer's radial-MLP
 * activations (about 12 F floats per undirected pair and layer, plus operand
 * copies) for the reverse pass; 1 = the reverse pass recomputes them, so the
 * workspace holds one layer's worth (for systems whose pair count presses on
 * memory).  Results are bitwise identical either way.
 * radial_table: 0 = the radial MLP and the radial projections run per pair;
 * n in [256, 16384] = both are functions of the pair distance alone, so they
 * are tabulated (FP64 values and d-derivatives, stored as FP32 cubic Hermite
 * coefficients per interval) at n points on [0, cutoff_upper] and
 * interpolated per pair; forces are the derivatives of the interpolated
 * energy.  The tables are built by tnet_radial_tables.  An inference mode:
 * weight gradients return UNSUPPORTED. */
typedef struct {
    int F, K, L, max_z;
    float cutoff_upper, cutoff_lower;
    int precision;
    int recompute_edges;
    int radial_table;
} tnet_model_desc;

typedef enum {
    TNET_OK = 0,
    TNET_ERR_ARG = 1,         /* bad argument (host) or bad batch vector (device) */
    TNET_ERR_CAPACITY = 2,    /* more pairs than the caller's capacity (device) */
    TNET_ERR_BOX = 3,         /* box not lower-triangular or narrower than 2*cutoff */
    TNET_ERR_NAN = 4,         /* non-finite position (device) */
    TNET_ERR_CUDA = 5,        /* a CUDA runtime call failed */
    TNET_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up */
    TNET_ERR_WORKSPACE = 7,   /* workspace too small or misaligned */
    TNET_ERR_Z = 8,           /* atomic number outside [0, max_z) (device) */
    TNET_ERR_UNSUPPORTED = 9, /* valid request this build does not implement */
    TNET_ERR_SKIN = 10        /* reserved (tnet_md_step rebuilds when an atom moves > skin/2) */
} tnet_status;

const char *tnet_status_string(int status);

/* Number of float32 values in the weight blob for this shape, or -1 for an
 * invalid shape.  Blob layout: the parameters below, each C-contiguous
 * float32, concatenated in this order with no padding.  Linear weights are
 * stored (out, in) so that y = W x + b; stacks [3] are indexed
 * p = 0 (I), 1 (A), 2 (S).
 *   emb        [max_z][F]       atomic-number embedding
 *   emb2_w     [F][2F], emb2_b [F]     pair embedding W_e [emb(z_i); emb(z_j)] + b_e
 *   dproj_w    [3][F][K], dproj_b [3][F]   radial projections f^p = W^p e(d) + b^p
 *   emb_ln_g   [F], emb_ln_b [F]           LayerNorm of the embedding norms
 *   emb_mlp1_w [2F][F], emb_mlp1_b [2F]
 *   emb_mlp2_w [3F][2F], emb_mlp2_b [3F]   per-atom scalar MLP (SiLU after each)
 *   emb_mix_w  [3][F][F]                   channel mixing of I, A, S (no bias)
 *   for l in 0..L-1:
 *     l{l}_mlp1_w [F][K],   l{l}_mlp1_b [F]
 *     l{l}_mlp2_w [2F][F],  l{l}_mlp2_b [2F]
 *     l{l}_mlp3_w [3F][2F], l{l}_mlp3_b [3F]  edge radial MLP (SiLU after each)
 *     l{l}_mix1_w [3][F][F]                   mixing before the messages
 *     l{l}_mix2_w [3][F][F]                   mixing after the tensor products
 *   out_ln_g   [3F], out_ln_b [3F]
 *   out_w      [F][3F], out_b [F]
 *   head1_w    [F/2][F], head1_b [F/2]
 *   head2_w    [1][F/2], head2_b [1]
 * Per-edge and per-atom 3F vectors are split channel-major: index c*3 + p. */
int64_t tnet_weights_count(const tnet_model_desc *desc);

/* Bytes of device workspace tnet_create needs for these limits (or -1 for
 * invalid arguments).  max_atoms: most atoms per call, max_systems: most
 * systems per call, max_pairs: the directed-pair capacity the caller will
 * pass to tnet_neighbors (also the most pairs tnet_energy_forces accepts). */
int64_t tnet_workspace_bytes(const tnet_model_desc *desc, int max_atoms, int max_systems,
                             int64_t max_pairs);

/* Create a context bound to the current CUDA device.  workspace: device
 * memory of at least tnet_workspace_bytes(...) bytes, 256-byte aligned,
 * owned by the caller and kept alive (and not used by anything else) until
 * tnet_destroy.  *out receives a host-side handle. */
int tnet_create(tnet_ctx **out, const tnet_model_desc *desc, int max_atoms, int max_systems,
                int64_t max_pairs, void *workspace, size_t workspace_bytes);
int tnet_destroy(tnet_ctx *ctx);

/* Neighbor search (Sec. 2.5.1): all ordered pairs (i, j), i != j, of atoms in
 * the same system with |r_i - r_j| < cutoff, where with periodic boundaries
 * the distance is that of the nearest image.  One cell list per system
 * (cells never mix systems); each system's cells are at least `cutoff`
 * wide, so a system smaller than two cutoffs is searched all-pairs.
 *   n_atoms, n_systems  counts (1 <= n_systems <= n_atoms is not required:
 *                       systems may be empty)
 *   pos      [N][3] float32
 *   batch    [N] int32 system index of each atom, non-decreasing, in
 *            [0, n_systems); NULL means every atom is in system 0
 *   box      [S][3][3] float32, rows a, b, c of each system's box, lower-
 *            triangular (a = (ax,0,0), b = (bx,by,0), c = (cx,cy,cz)),
 *            rectangular or triclinic, reduced or not (Sec. 2.5.1: periodic
 *            boundary conditions with rectangular and triclinic boxes);
 *            NULL means no periodicity.  Each perpendicular width must be
 *            >= 2*cutoff (else BOX); the nearest image (remove c, then b,
 *            then a) is then exact for every pair within the cutoff.
 *   cutoff   Angstrom (> 0); a pair is kept when d < cutoff
 * Output (receiver-sorted CSR; within a row, columns ascend):
 *   row_ptr  [N+1] int32   row_ptr[0] = 0, row i holds the j of pairs (i, j)
 *   col      [cap] int32
 *   n_pairs_dev  [1] int64 number of pairs found (also when > cap)
 * If the pairs exceed cap, status CAPACITY is set, *n_pairs_dev still holds
 * the number of pairs found, row_ptr holds the exact row offsets clamped to
 * cap (so no reader of the truncated list leaves col; the rows that end at
 * or below cap are complete), col is filled only below cap, and the caller
 * must enlarge col to *n_pairs_dev and call again.  cap must not exceed the
 * context's max_pairs. */
int tnet_neighbors(tnet_ctx *ctx, int n_atoms, int n_systems, const float *pos,
                   const int32_t *batch, const float *box, float cutoff, int32_t *row_ptr,
                   int32_t *col, int64_t cap, int64_t *n_pairs_dev, int32_t *status_dev,
                   tnet_stream_t stream);

/* Energy and forces (Sec. 2, Fig. 1; TensorNet Sec. 2.1.1): per-system
 * energies E_s = sum over atoms of the system of the per-atom output, and
 * forces F_i = -dE/dr_i computed by a hand-written reverse pass.
 *   weights  flat blob, tnet_weights_count floats (layout above)
 *   z [N] int32 atomic numbers in [0, max_z); pos, batch, box as in
 *   tnet_neighbors; row_ptr/col: a symmetric pair list from tnet_neighbors
 *   built with a cutoff >= cutoff_upper (pairs at d >= cutoff_upper
 *   contribute nothing, so a list with a skin is valid)
 *   energy_seed [S] float32 or NULL: forces and weight gradients are those of
 *            sum_s seed_s E_s (NULL: all ones)
 *   energy   [S] float64 output
 *   forces   [N][3] float32 output, or NULL to skip the reverse pass
 *   grad_weights  [tnet_weights_count] float32 output (overwritten) or NULL.
 * Results do not depend on the order of columns within a row beyond float
 * rounding; with the CSR of tnet_neighbors they are deterministic. */
int tnet_energy_forces(tnet_ctx *ctx, const float *weights, int n_atoms, int n_systems,
                       const int32_t *z, const float *pos, const int32_t *batch,
                       const float *box, const int32_t *row_ptr, const int32_t *col,
                       const float *energy_seed, double *energy, float *forces,
                       float *grad_weights, int32_t *status_dev, tnet_stream_t stream);

/* Radial-function tables (contexts with radial_table = n > 0).  The radial
 * projections f(d) and every layer's filter g(d) (TensorNet Sec. 2.1.1: the
 * expnorm basis, the cosine cutoff and the radial MLP) depend on the pair
 * distance and the weights alone.  This call evaluates them, with their
 * d-derivatives, from `weights` at the n points d_k = k cutoff_upper/(n-1),
 * in FP64, and stores each interval's cubic Hermite polynomial (coefficients
 * formed in FP64, kept as FP32) in the context's workspace;
 * tnet_energy_forces and tnet_md_step then interpolate them and do not read
 * the radial weights.  Call it again
 * whenever those weights change.  Before the first call, tnet_energy_forces
 * and tnet_md_step of a table-mode context return TNET_ERR_ARG.  Stream
 * ordered (the tables are ready for work enqueued after it on `stream`);
 * graph-capturable.  Contexts without tables: TNET_ERR_ARG. */
int tnet_radial_tables(tnet_ctx *ctx, const float *weights, tnet_stream_t stream);

/* Molecular dynamics (the paper's MD use, Sec. 3 "Molecular Simulations";
 * one step = one energy evaluation plus one force backward pass): n_steps
 * velocity-Verlet steps of one system with time step dt_fs:
 *   v += dt/2 F/m; x += dt v; [neighbor list at cutoff_upper + skin: every
 *   rebuild_every steps, and in any step where an atom has moved more than
 *   skin/2 since the last rebuild]; F = forces(x); v += dt/2 F/m.
 * Forces in eV/A and masses in amu are converted with
 * 1 eV/(A amu) = 9.64853321e-3 A/fs^2.
 *   inv_mass [N] float32 1/m in 1/amu; pos, vel [N][3] float32 updated in
 *   place (vel in A/fs); box [1][3][3] or NULL
 *   e_kin, e_pot [n_steps] float64 outputs: kinetic and potential energy
 *   after each step
 * The steps run as replays of a CUDA graph of rebuild_every steps that the
 * context captures on first use and re-captures when a pointer, count or
 * parameter changes.  The displacement test runs on the device in every
 * step; a step that does not rebuild runs the neighbor kernels as no-ops, so
 * the list always holds every pair within cutoff_upper and the trajectory
 * does not depend on skin or rebuild_every.
 * Requires max_pairs >= the pairs within cutoff_upper + skin. */
int tnet_md_step(tnet_ctx *ctx, const float *weights, int n_atoms, const int32_t *z,
                 const float *inv_mass, float *pos, float *vel, const float *box, float dt_fs,
                 float skin, int rebuild_every, int n_steps, double *e_kin, double *e_pot,
                 int32_t *status_dev, tnet_stream_t stream);

/* Number of neighbor-list builds (periodic and displacement-triggered,
 * including the initial one) of the last tnet_md_step call on this context.
 * Synchronous: waits for the device.  count: host pointer. */
int tnet_md_rebuilds(tnet_ctx *ctx, int64_t *count);

/* Copy of the neighbor list tnet_md_step keeps in the context (CSR at
 * cutoff_upper + skin, built at the last rebuild of the last call), stream-
 * ordered on `stream`: row_ptr [n_atoms+1] and col [min(n_pairs, cap)] device
 * buffers of the caller, n_pairs a device int64. */
int tnet_md_neighbor_list(tnet_ctx *ctx, int n_atoms, int32_t *row_ptr, int32_t *col, int64_t cap,
                          int64_t *n_pairs, tnet_stream_t stream);

/* ---- allocation-free neighbor search (no counterpart in the paper) -------
 * For callers that cannot allocate device memory (code inside another
 * framework's memory pool or a real-time loop that forbids cudaMalloc after
 * start-up, or plain C callers with no allocator): the same search as
 * tnet_neighbors, with the same arguments and outputs but no context, its
 * scratch held in a file-scope __device__ array of 2 MiB that every GPU
 * loading the library keeps until the process exits.  The caller still
 * passes all inputs and outputs.
 * Limits: n_atoms <= 16384 and n_systems <= 1024; larger requests return
 * TNET_ERR_WORKSPACE at once (nothing is enqueued).  No cudaMalloc, cudaFree
 * or allocating library call is made.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress), so make that first call
 * before any stream capture.  All calls share the array: calls whose GPU
 * work overlaps (different streams or threads) race; calls ordered on one
 * stream are safe.  Each call lays the array out for its own n_atoms and
 * n_systems and zeroes what must start at zero, so its cost follows the
 * input, not the limits. */
int tnet_neighbors_noalloc(int n_atoms, int n_systems, const float *pos, const int32_t *batch,
                           const float *box, float cutoff, int32_t *row_ptr, int32_t *col, int64_t cap,
                           int64_t *n_pairs_dev, int32_t *status_dev, tnet_stream_t stream);

/* ---- testing (no counterpart in the paper) --------------------------------
 * C[M][N] = A[M][K] * B[N][K]^T on the tensor cores (tcgen05, BF16 inputs,
 * FP32 accumulation), the GEMM engine of the BF16 precision mode, exposed so
 * that tests can check it against a library matmul.  A, B bf16 K-major
 * device arrays, C float32 [M][N]; K a multiple of 8, N a multiple of 4 and
 * <= 512.  Bounded in-kernel waits report TNET_ERR_TIMEOUT in *status_dev. */
int tnet_debug_tc_gemm(int M, int N, int K, const void *A, const void *B, float *C, int32_t *status_dev,
                       tnet_stream_t stream);
/* The same in 3xTF32: A [M][K], B [N][K] float32; B_split is caller scratch
 * of 2*N*K floats that receives B's TF32 split (high parts, then the rounded
 * remainders; A's split is formed inside the kernel); K a multiple of 4, N a
 * multiple of 4 and <= 512. */
int tnet_debug_tc_gemm_f32(int M, int N, int K, const float *A, const float *B, float *B_split, float *C,
                           int32_t *status_dev, tnet_stream_t stream);
/* Either of the two above (x3 = 1: 3xTF32, B_split as there; x3 = 0: BF16,
 * B_split unused) with the CTAs in thread-block clusters of `cluster` (1, 2
 * or 4) that share each weight stage through TMA multicast, the form the
 * library uses for one-class GEMMs; TNET_ERR_ARG for another cluster size or
 * the shape errors above.  A tile whose rows do not split into whole 8-row
 * groups per CTA runs without clusters. */
int tnet_debug_tc_gemm_cluster(int M, int N, int K, int x3, int cluster, const void *A, const void *B,
                               float *B_split, float *C, int32_t *status_dev, tnet_stream_t stream);
/* Test of the failure path of the tensor-core kernel (no counterpart in the
 * paper): the 3xTF32 GEMM above with its MMA issuer told to issue nothing and
 * every mbarrier wait bounded by spin_limit (>= 1) tries instead of the
 * library's limit.  The loads land, nothing consumes them, the bounded waits
 * run out: the kernel records TNET_ERR_TIMEOUT in *status_dev, waits for its
 * own copies, frees its tensor memory and returns, leaving the context
 * usable.  C is not written.  Returns TNET_ERR_ARG for spin_limit 0 or the
 * shape errors of tnet_debug_tc_gemm_f32. */
int tnet_debug_tc_gemm_timeout(int M, int N, int K, const float *A, const float *B, float *B_split, float *C,
                               uint32_t spin_limit, int32_t *status_dev, tnet_stream_t stream);

/* ---- tuning (no counterpart in the paper) ---------------------------------
 * Launch-shape knobs of a context: grid sizes, GEMM column tiles and whether
 * kernels use programmatic dependent launch (the next kernel is scheduled
 * while the previous one drains).  Every value is valid on any input; the
 * choice only changes speed.  Knob k takes
 * one of tnet_tuning_candidates(k, ...) (the count is returned; values are
 * written up to max).  tnet_set_tuning rejects values outside the candidate
 * lists.  A new context starts from fixed defaults, with programmatic launch
 * on only when max_atoms <= 1024.  An autotuner times the candidates on a
 * real input (as CUDA-graph replays) and sets the fastest
 * (paper_2402_17660_gb300.tnet.autotune). */
int tnet_tuning_knobs(void);
const char *tnet_tuning_name(int knob);
int tnet_tuning_candidates(int knob, int32_t *values, int max);
int tnet_get_tuning(tnet_ctx *ctx, int32_t *knobs, int n);
int tnet_set_tuning(tnet_ctx *ctx, const int32_t *knobs, int n);

/* ---- instrumentation (no counterpart in the paper; used by the benchmark) */

/* Number of CUDA kernels the library has enqueued in this process (all
 * contexts, host-side count; a launch captured into a graph counts once, at
 * capture time). */
int64_t tnet_launch_count(void);

/* Stage profiler.  tnet_profile(ctx, 1) clears and starts recording CUDA
 * events around each stage of later calls on this context (not while the
 * stream is being captured); tnet_profile(ctx, 0) stops.  tnet_profile_read
 * synchronises on the recorded events and returns, for tags 0..ntags-1,
 * the summed milliseconds and the number of recorded stage instances.
 * tnet_profile_tag(t) names tag t, or returns NULL past the last tag. */
int tnet_profile(tnet_ctx *ctx, int enable);
int tnet_profile_read(tnet_ctx *ctx, int ntags, float *ms, int64_t *count);
const char *tnet_profile_tag(int tag);

#ifdef __cplusplus
}
#endif
#endif /* TNET_H */
