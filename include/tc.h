/*
 * tc.h -- C ABI of libtc, a single-GPU (sm_103a) treecode force library.
 *
 * The treecode (Barnes-Hut) of the paper, Sec. 3.1: the bodies are put in an
 * oct-tree by recursively dividing space into 8 sub-cubes until a cube holds
 * no more than a threshold of bodies; each cell stands for its bodies by
 * their total mass at their centre of mass; the force on a body is found by
 * walking the tree from the root, adding a cell to the body's interaction
 * list when it is distant enough and descending into its children
 * otherwise, then summing the list with F = G m_a m_b / r^2; finally every
 * body updates its position and velocity from the force.  The paper spends
 * upwards of 90% of the cycles in the force summation (Sec. 1, Sec. 3.2).
 *
 * Conventions for every function below
 *   - Return value: TC_OK (0) or a negative TC_E* code; tc_last_error() gives
 *     a one-line reason.  The library never aborts and never prints.
 *   - Pointers: any pointer argument may be host or device memory (unified
 *     addressing); the library copies inputs into its own device buffers and
 *     the caller keeps ownership of everything it passes.
 *   - Layouts: positions, velocities and accelerations are n x 3 float32,
 *     row-major (x, y, z per body), in the caller's (original) body order;
 *     masses are n float32.
 *   - Streams: all work is enqueued on the context's stream.  Calls that only
 *     enqueue return before the GPU work ends; calls that hand data back
 *     (tc_get_*, tc_diag, tc_direct, tc_sync) synchronise the stream and also
 *     report device-side errors (TC_EDEVICE) raised by earlier work.
 *   - Not thread-safe per context; distinct contexts are independent.
 */
#ifndef TC_H
#define TC_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TC_OK 0
#define TC_EINVAL (-1)  /* invalid argument (n < 1, leaf_max out of range, theta < 0, eps <= 0, NaN/Inf, mass <= 0) */
#define TC_ENOMEM (-2)  /* device allocation failed (or the TC_ALLOC_CAP_BYTES cap was hit) */
#define TC_ESTATE (-3)  /* call out of order (forces before build, step before forces) */
#define TC_EDEVICE (-4) /* a kernel raised its error word (walk stack overflow, ...) */
#define TC_ECUDA (-5)   /* a CUDA runtime call failed */

typedef struct tc_ctx tc_ctx;

/* Tuning of the force phase (the autotuner's output).
 *   gmax      bodies per group walk: 1..32, 64 or 128 (one, two or four
 *             bodies per lane); gmax = 1 gives every body its own walk and
 *             list (the paper's per-body lists; one lane in 32 sums)
 *   warps     warps per block of the walk kernel, 1..4
 *   precise   1: cell-relative coordinates for cell sources and compensated
 *             (TwoSum) accumulation across list tiles; 0: absolute float32
 *             coordinates and plain accumulation
 *   want_pot  1: also compute the potential (tc_get_acc's pot, tc_diag's PE)
 *   verify    1: record per-group list lengths and hashes (tc_get_lists)
 *   stack     walk stack entries per warp (shared memory), 64..8192
 *   blocks_per_sm  0 = as many as fit, else a cap
 *   quad      1: also reduce the cells' second moments about the centre of
 *             mass (FP32, within (leaf_max + 128) 2^-25 M s^2; the learned
 *             correction's features and the quadrupole walk, tc_get_nodes'
 *             quad); 0: mass and centre of mass only
 *   tile      interaction-list entries summed per shared-memory tile: 64,
 *             128 or 256
 *   graph     1: tc_ctx_step replays one captured CUDA graph per step (the
 *             whole step -- kick, drift, rebuild, walk, kick -- with no host
 *             synchronisation; with phase timing on, the walk and the
 *             closing kick follow the graph as timed launches); 0: the same
 *             launches issued one by one
 *   learned   1: add the learned far-field correction of tc_mlp_set /
 *             tc_mlp_train to the walk (needs precise = 1, want_pot = 0,
 *             quad = 1, quadrupole = 0)
 *   quadrupole 1: every accepted cell adds its quadrupole term to its
 *             monopole (second-order expansion of the softened potential
 *             about the centre of mass; needs precise = 1, quad = 1)
 *   classes   1: with gmax 64 or 128 the walk runs one launch per group
 *             size class (the largest on the calling stream, the others
 *             beside it on a stream of the context's, joined back before the
 *             call returns its work to the stream): a group of at most 32 bodies is
 *             summed one body per lane, one of at most 64 two per lane, a
 *             larger one four (the default); 0: one launch, gmax / 32
 *             bodies per lane for every group.  Lists and forces are the
 *             same in both.
 *   split     1: the monopole walks (learned = 0, quadrupole = 0) run with
 *             the tree walk and the force loop on different warps: a
 *             producer warp walks and fills a ring of list tiles in shared
 *             memory, a consumer warp sums them (the default); the learned
 *             walk stays on one warp per group with the network evaluated
 *             inside the walk.  2: the learned walk also splits, its band
 *             cells recorded by the producers and the network run on all of
 *             them after the walk.  0: every warp walks and sums its own
 *             groups.  Same lists; the sums take the tiles in another order
 *             (rounding-level differences). */
typedef struct {
    int32_t gmax;
    int32_t warps;
    int32_t precise;
    int32_t want_pot;
    int32_t verify;
    int32_t stack;
    int32_t blocks_per_sm;
    int32_t quad;
    int32_t tile;
    int32_t graph;
    int32_t learned;
    int32_t quadrupole;
    int32_t classes;
    int32_t split;
} tc_config;

/* Create a context on the current CUDA device.  `cuda_stream` is a
 * cudaStream_t (NULL = the legacy default stream); it must outlive the
 * context. */
int tc_create(tc_ctx **ctx, void *cuda_stream);
void tc_destroy(tc_ctx *ctx);
int tc_set_config(tc_ctx *ctx, const tc_config *cfg);
int tc_get_config(tc_ctx *ctx, tc_config *cfg);
int tc_set_stream(tc_ctx *ctx, void *cuda_stream);

/* Tree construction (Sec. 3.1): copies pos (n x 3) and mass (n), builds the
 * root cube, Morton keys (stable sort), the oct-tree with leaf threshold
 * leaf_max (a cube is divided while it holds more than leaf_max bodies,
 * down to level 21), the cells' masses and centres of mass (bottom-up sums
 * as pairs of floats, FP64-class: within 1e-12 of the exact sums; results
 * stored in FP64) and the body groups.  1 <= n < 2^31, 1 <= leaf_max <= 4096, masses > 0.
 * Velocities are reset to zero when n changes.  Synchronises with the
 * device part-way (to report invalid input and size the node table); the
 * rest is enqueued. */
int tc_ctx_build(tc_ctx *ctx, const float *pos, const float *mass, int64_t n, int leaf_max);

/* A batch of nsys independent systems in one context (bodies of system s are
 * pos/mass rows [offsets[s], offsets[s+1]); offsets has nsys + 1 entries,
 * offsets[0] = 0, every system holds at least one body, 1 <= nsys <= 65536).
 * Each system gets its own root cube and tree (one forest); forces act only
 * within a system; one walk launch and one step graph serve all systems.
 * tc_ctx_build is the batch of one system. */
int tc_ctx_build_batch(tc_ctx *ctx, const float *pos, const float *mass, const int64_t *offsets,
                       int64_t nsys, int leaf_max);

/* Velocities (n x 3) for tc_ctx_step; copied. */
int tc_ctx_set_velocity(tc_ctx *ctx, const float *vel);

/* Force phase (Sec. 3.1, Sec. 3.2): for every body group, walk the tree from
 * the root with the opening test "accept a cell of side s whose centre of
 * mass is at distance d from the group's bounding box iff it holds none of
 * the group's bodies and s < theta * d", then sum the accepted cells and the
 * bodies of opened leaves with the Plummer-softened force law
 *   a_i = G sum_j m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^(3/2).
 * theta >= 0 (0 = direct summation through the tree), eps > 0.  Results stay
 * on the device (tc_get_acc).  Enqueue only. */
int tc_ctx_forces(tc_ctx *ctx, float theta, float eps, float G);

/* One kick-drift-kick leapfrog step of length dt with the last theta, eps,
 * G: v += a dt/2; x += v dt; rebuild the tree; forces; v += a dt/2 (the
 * paper's "each body updates its position and velocity", Sec. 3.1).  Needs
 * a prior tc_ctx_forces on the current positions.  Enqueue only: the rebuild
 * reuses the node table sized by the last tc_ctx_build / tc_set_state (with
 * 50% headroom); a tree that outgrows it stops the step on the device and
 * the next synchronising call reports TC_EDEVICE. */
int tc_ctx_step(tc_ctx *ctx, float dt);

/* Accelerations (n x 3) and, if pot != NULL and want_pot was set, the
 * potential (n) of the last force phase, original body order. */
int tc_get_acc(tc_ctx *ctx, float *acc, float *pot);

/* Current positions / velocities (n x 3 each; either may be NULL). */
int tc_get_state(tc_ctx *ctx, float *pos, float *vel);
/* Replace positions and velocities (n x 3 each, n of the last build) and
 * rebuild the tree; forces must be recomputed before the next step. */
int tc_set_state(tc_ctx *ctx, const float *pos, const float *vel);

/* Sizes of the last build: bodies, nodes, groups (any may be NULL). */
int tc_get_sizes(tc_ctx *ctx, int64_t *n, int64_t *nnodes, int64_t *ngroups);

/* Verification exports of the last build (any pointer may be NULL).
 *   perm[n]      Morton position -> original index
 *   keys[n]      sorted 63-bit Morton keys
 * Node table in breadth-first order (by level, then first body), nnodes long:
 *   level, prefix (3*level-bit Morton prefix), first, count, child_first
 *   (-1 for a leaf), nchild, mass, com (3 per node, absolute), quad (6 per
 *   node: xx, xy, xz, yy, yz, zz second moments about the centre of mass;
 *   needs quad = 1 in the configuration, else TC_ESTATE).
 * Groups, ngroups long: gfirst, gcount, gref (reference cube index). */
int tc_get_tree(tc_ctx *ctx, uint32_t *perm, uint64_t *keys);
int tc_get_nodes(tc_ctx *ctx, int32_t *level, uint64_t *prefix, int32_t *first, int32_t *count,
                 int32_t *child_first, int32_t *nchild, double *mass, double *com, double *quad);
int tc_get_groups(tc_ctx *ctx, int32_t *gfirst, int32_t *gcount, int32_t *gref);
/* Root cube of the last build (system 0): out5 = {c0x, c0y, c0z, L, h}. */
int tc_get_cube(tc_ctx *ctx, double *out5);
/* Number of systems and their root cubes (nsys x 5, as tc_get_cube). */
int tc_get_systems(tc_ctx *ctx, int64_t *nsys, double *cubes);

/* List-export mode: the interaction list of one group (the paper's
 * ComputeForces receives a body with its list, Sec. 3.2) at opening angle
 * theta on the current tree: the accepted cells and the opened leaves as
 * breadth-first node indices (tc_get_nodes), in the walk's discovery order.
 * cells / leaves (host or device, nullable) receive at most cap entries
 * each; *ncells / *nleaves the full lengths.  With gmax = 1 a group is one
 * body and this is its per-body list.  The context's forces and list totals
 * are left as they were.  TC_EINVAL for a group outside [0, G). */
int tc_get_group_list(tc_ctx *ctx, int64_t group, float theta, int32_t *cells, int32_t *leaves, int64_t cap,
                      int64_t *ncells, int64_t *nleaves);

/* Per-group list lengths of the last force phase (needs verify = 1):
 * accepted cells, bodies of opened leaves, order-independent hash of the
 * accepted cells and opened leaves; and totals over groups of group size x
 * list length: interactions = cells + bodies, cells = body-cell terms,
 * bodies = body-body terms.  Any pointer may be NULL. */
int tc_get_lists(tc_ctx *ctx, int32_t *ncell, int32_t *nbody, uint64_t *hash,
                 int64_t *interactions, int64_t *cells, int64_t *bodies);

/* FP64 diagnostics of the current state: out8 = {kinetic energy,
 * potential energy 1/2 sum m_i pot_i (needs want_pot), momentum x, y, z,
 * angular momentum x, y, z}. */
int tc_diag(tc_ctx *ctx, double *out8);

/* Direct O(N * ns) summation for bodies idx[0..ns) (original indices) over
 * all n bodies of the current state: acc (ns x 3) and pot (ns, nullable),
 * FP32 terms, FP64 accumulation.  The accuracy reference of the treecode. */
int tc_direct(tc_ctx *ctx, const int64_t *idx, int64_t ns, float eps, float G, double *acc,
              double *pot);

/* Phase timers.  tc_set_timing(ctx, 1) starts recording CUDA events on the
 * context's stream around the build, the walk + force kernel and the
 * leapfrog updates (and clears earlier records).  tc_get_timings
 * synchronises and returns out6 = {build ms, walk ms, update ms (sums over
 * the calls since the last tc_set_timing / tc_get_timings), kernels launched
 * by this process's libtc since then (a replayed step graph counts its
 * kernels), kernels launched in total, kernels in one step graph}, then
 * clears the records.  In graph mode with timing on, a step's graph holds
 * kick + drift + rebuild (timed as "build") and the walk and closing kick
 * are launched after it, each bracketed by events. */
int tc_set_timing(tc_ctx *ctx, int on);
int tc_get_timings(tc_ctx *ctx, double *out6);

/* Direct summation with no device allocation (no counterpart in the paper;
 * the same sums as tc_direct).  For callers that cannot let a library call
 * cudaMalloc -- a framework whose caching allocator already owns the
 * device's memory budget, or a latency-critical loop that cannot afford the
 * implicit synchronisation of cudaMalloc/cudaFree.  Nothing is allocated:
 * the inputs are read where they are, the outputs written where they are,
 * and the only scratch (per-slice partial sums) lives in a fixed 4 MiB
 * array that every GPU loading libtc holds until the process exits.
 *   pos (n x 3 float32), mass (n float32), idx (ns int64, original
 *   indices in [0, n)), acc (ns x 3 float64), pot (ns float64, nullable):
 *   memory the current device reaches in place -- its own device memory,
 *   managed memory or mapped pinned host memory.  Host pageable memory and
 *   another device's memory are rejected (TC_EINVAL): the first would need
 *   staging, the second may not be peer-mapped.  The C ABI cannot see
 *   element types or array lengths: buffers shorter than stated, or of
 *   other types, are read or written out of bounds.  An index outside
 *   [0, n) yields NaN for that target (it is never dereferenced).
 *   1 <= ns <= 8192 (the scratch's capacity; more is rejected with
 *   TC_EINVAL), 1 <= n < 2^31, eps > 0.
 *   stream: cudaStream_t of the current device for the two kernels
 *   (NULL = legacy default); the call only enqueues.  A CUDA error already
 *   pending when the call starts is returned as TC_ECUDA (and left
 *   pending) before anything is launched.
 * The first call on a device looks up the device address of the scratch
 * array (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls on a device share the scratch: calls whose work
 * overlaps on the GPU (different streams, no ordering) race and give
 * wrong results.  Errors: tc_last_error(NULL) gives the reason (while the
 * implicit default context has no error of its own pending). */
int tc_direct_static(const float *pos, const float *mass, int64_t n, const int64_t *idx, int64_t ns,
                     float eps, float G, double *acc, double *pot, void *cuda_stream);

/* Fast multipole method on the current tree (Sec. 5 names the FMM as the
 * treecode's O(N) successor and gives no formulation; this is the reading
 * implemented):
 *   expansion centres  every cell's centre of mass c_X (the build's FP64
 *                      reduction); its multipole is the monopole M_X;
 *   radii              r_X bounds the distance of X's bodies from c_X: a
 *                      leaf's farthest body, above the farthest child
 *                      sphere, max over children of |c_child - c_X| +
 *                      r_child (FP64, rounded to FP32 for the test);
 *   local expansions   third order about c_B: near B the field is
 *                      a(x) = L0 + L1 dx + (1/2) L2 dx dx + (1/6) L3 dx dx dx,
 *                      dx = x - c_B, L1 the field's Jacobian, L2 and L3 its
 *                      second and third derivatives (FP32, symmetric
 *                      storage);
 *   acceptance         distinct cells A, B with r_A + r_B < theta |c_A - c_B|,
 *                      tested in FP32;
 *   traversal          dual, from (root, root): a cell paired with itself
 *                      splits into every (child, child) pair (a leaf: P2P
 *                      within it); an accepted pair is an M2L from A to B;
 *                      two leaves are a P2P; otherwise B is split when it is
 *                      internal and (A is a leaf or r_B >= r_A), else A;
 *   M2L (A -> B)       the Plummer-softened field G M_A d / rho^3 of A's
 *                      monopole, d = c_A - c_B, rho^2 = |d|^2 + eps^2, and
 *                      its first three derivatives, added to L(B);
 *   L2L                parents before children: L(child) += L(parent)
 *                      moved to the child's centre (exact for a cubic);
 *   L2P, P2P           every body of a leaf gets its leaf's expansion and
 *                      the softened direct sum over the bodies of every leaf
 *                      P2P-paired with it (compensated FP32 summation).
 * Every ordered pair of bodies is counted exactly once, through one M2L or
 * one P2P.  theta >= 0 (0: every pair is P2P, the direct sum), eps > 0.
 * The accelerations replace the context's (tc_get_acc; no potential), and
 * tc_ctx_step refuses them (TC_ESTATE): a step integrates with the treecode.
 * Synchronises (it reads the tree's level ranges and checks its scratch).
 * Scratch is kept in the context and grows as needed: a pass whose lists
 * outgrew it is rerun.  TC_EDEVICE when a cell's refinement stack overflows
 * (2048 sources; theta far below 0.2 on strongly clustered bodies). */
int tc_ctx_fmm(tc_ctx *ctx, float theta, float eps, float G);
/* Pair counts of the last tc_ctx_fmm (M2L, P2P, self pairs of leaves
 * included) and two order-independent hashes of the pair sets: the sums
 * over pairs of splitmix64((A << 32) ^ B), A source and B target
 * breadth-first node indices (tc_get_nodes).  Any pointer may be NULL;
 * hash2 receives {M2L hash, P2P hash} and needs verify = 1 in the
 * configuration of that pass (else TC_ESTATE). */
int tc_get_fmm_stats(tc_ctx *ctx, int64_t *m2l, int64_t *p2p, uint64_t *hash2);
/* The same per target cell (nnodes entries each, host memory, any may be
 * NULL): M2L and P2P pairs whose target is the cell, and their hashes
 * (verify = 1 in the configuration of that pass, else TC_ESTATE). */
int tc_get_fmm_pairs(tc_ctx *ctx, int64_t *nm2l, int64_t *np2p, uint64_t *hm2l, uint64_t *hp2p);

/* Autotuner: times the walk + force kernel for every group size (32, 64,
 * 128), list tile (64, 128, 256) and warps per block (2, 4) on the current
 * bodies (reps timed runs each, the fastest kept), sets the best and returns
 * it with its time in ms.  When the environment variable TC_AUTOTUNE_CACHE
 * names a file, results are looked up there first and appended after a
 * search (key: N, systems, leaf, theta, eps, precision, potential). */
int tc_autotune(tc_ctx *ctx, float theta, float eps, float G, int reps, tc_config *best, double *best_ms);

/* ---- Learned far-field correction (a growth of the method; the paper
 * describes only the monopole walk).  An MLP 13 -> 64 -> 64 -> 3 (ReLU)
 * predicts the error of a cell's monopole term at a point x.  With d =
 * com - x, r = |d|, s the cell side and M its mass:
 *   factor F = G M s^2 / r^4   (the scale of the quadrupole term)
 *   label    = (a_exact - a_mono) / F
 * where a_exact is the softened direct sum over the cell's bodies and a_mono
 * the softened monopole; features (13): d/s (3), s/r, eps/s, log2(count),
 * M / (system mass), Q_ab / (M s^2) (xx, xy, xz, yy, yz, zz), Q the second
 * moments about the centre of mass.  BF16 operands on the tensor cores, FP32
 * accumulation and master weights.  In the walk (learned = 1) every
 * accepted cell holding two or more bodies with s >= band * d (d the
 * distance from its centre of mass to the group's box) is evaluated once
 * per group at the centre of the group's box, and F * label is added to
 * every body of the group.
 *
 * A model is TC_MLP_NMODEL floats: the parameters W1[13][64], b1[64],
 * W2[64][64], b2[64], W3[64][3], b3[3] (W[i][j]: input i to output j), then
 * 13 feature means, 13 feature scales (features enter the network as
 * (f - mean) * scale) and 3 output scales (label = output * scale).
 * Array arguments may be host or device memory; the calls below return when
 * their results are in place (they synchronise the context's stream). */
#define TC_MLP_NPARAM (13 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3)
#define TC_MLP_NMODEL (TC_MLP_NPARAM + 13 + 13 + 3)
/* Set the model (non-finite values: TC_EINVAL) and the band (>= 0). */
int tc_mlp_set(tc_ctx *ctx, const float *model, float band);
/* Read the model and band back (TC_ESTATE without a model); both nullable. */
int tc_mlp_get(tc_ctx *ctx, float *model, float *band);
/* labels (n x 3) of raw features X (n x 13) under the current model */
int tc_mlp_forward(tc_ctx *ctx, const float *X, int64_t n, float *Y);
/* loss (1/n) sum w_i |output_i - T_i / scale|^2 over the n pairs (W: n
 * weights >= 0, NULL for all 1) and its gradient (TC_MLP_NPARAM, packed like
 * the parameters) under the current model; grad and loss nullable */
int tc_mlp_loss_grad(tc_ctx *ctx, const float *X, const float *T, const float *W, int64_t n, float *grad,
                     float *loss);
/* Train a fresh model (weights and biases uniform in +-1/sqrt(fan-in), from
 * a counter-based generator keyed by seed; feature means/scales and output
 * RMS from the data) on n >= 16 pairs (X n x 13 features, T n x 3 labels)
 * with Adam, learning rate lr decayed along a cosine over all steps,
 * mini-batches of `batch` (>= 16) in a fresh seeded order each pass,
 * `epochs` passes; sets it as the context's model with the given band.
 * Loss weights: weight_mode TC_MLP_WEIGHTS takes W (n, >= 0; NULL for all
 * 1) as the weights; TC_MLP_FACTORS takes W as the pairs' label factors F
 * (tc_mlp_pairs) and weights each pair by F^2 / mean(F^2), which makes the
 * loss the mean squared error of the corrected acceleration.  Everything,
 * the data's statistics included, is computed on the device.  losses[epochs]
 * (nullable) gets the mean mini-batch loss of each pass. */
#define TC_MLP_WEIGHTS 0
#define TC_MLP_FACTORS 1
int tc_mlp_train(tc_ctx *ctx, const float *X, const float *T, const float *W, int32_t weight_mode, int64_t n,
                 int epochs, int batch, float lr, uint64_t seed, float band, float *losses);
/* Training pairs generated by the method itself: a walk at theta over the
 * current bodies emits, with probability prob (seeded), every accepted cell
 * holding two or more bodies with s >= band * d, paired with a body of the
 * group; features at that body, the exact label and the factor F (G = 1).
 * Outputs (any nullable except npairs): X (max_pairs x 13), T (max_pairs x
 * 3), F (max_pairs), body (original index), node (breadth-first index);
 * *npairs = pairs written (at most max_pairs).  The pairs come in one order
 * (by body position in the tree, then node), whatever the order the walk
 * emitted them in, so the same bodies, theta, band, prob and seed give the
 * same pairs in the same order -- as long as no more than max_pairs are
 * emitted (past the cap, which pairs are kept depends on the walk's
 * schedule).  Needs quad = 1; overwrites the context's accelerations. */
int tc_mlp_pairs(tc_ctx *ctx, float theta, float eps, float band, float prob, uint64_t seed, int64_t max_pairs,
                 float *X, float *T, float *F, int64_t *body, int64_t *node, int64_t *npairs);
/* corrections evaluated by learned walks since the last call */
int tc_mlp_evals(tc_ctx *ctx, int64_t *evals);

/* Measured FP32 throughput of the current device in TFLOP/s (FMA = 2
 * flops): a grid of 8 x 256-thread blocks per SM, each thread running 8
 * independent chains of scalar (paired = 0) or paired f32x2 (paired = 1)
 * fused multiply-adds; best of three timed launches. */
int tc_probe_fp32(int paired, double *tflops);

/* Measured throughput of the walk's force loop alone, in TFLOP/s at 20
 * flops per body-source interaction: 4 blocks of 4 warps per SM (the walk's
 * occupancy), each warp summing a 128-entry list tile in shared memory
 * against two bodies per lane through the walk's own flush (paired FP32
 * loop, SFU rsqrt, compensated accumulation), 4096 times; best of three
 * timed launches.  No tree, no walk: the ceiling of the loop as written. */
int tc_probe_force(double *tflops);

/* Self-test of the failure path: runs one radix pass tile whose predecessor
 * never publishes, so its bounded look-back gives up (after about a second)
 * instead of waiting forever.  *err_bits receives the device error word it
 * set (8: a bounded device wait gave up), *elapsed_ms (nullable) the time
 * the kernel took.  Uses its own buffers and stream on the current device;
 * returns TC_OK when the kernel completed (whatever it reported). */
int tc_selftest_bounded_wait(int32_t *err_bits, double *elapsed_ms);

/* Wait for the context's stream; report device errors. */
int tc_sync(tc_ctx *ctx);

/* Reason of the last failure of this context (NULL: the default context). */
const char *tc_last_error(tc_ctx *ctx);

/* The three calls of the treecode on an implicit default context (created
 * on first use on the current device and the legacy default stream). */
int tc_build(const float *pos, const float *mass, int64_t n, int leaf_max);
int tc_forces(float theta, float eps, float G);
int tc_step(float dt);
tc_ctx *tc_default(void);

#ifdef __cplusplus
}
#endif
#endif
