// tc_internal.cuh -- device-side data layout and launchers of the treecode
// library (CUDA, sm_103a).  Internal to libtc.so; the public C ABI is
// include/tc.h.
//
// A context holds a batch of S >= 1 independent systems whose bodies are
// concatenated (system s owns bodies [off_s, off_s+1) in the caller's order
// and the same positions in Morton order).  Every system has its own root
// cube and its own tree; the trees form one forest in one node table, and
// one walk launch serves the groups of every system.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tc {

constexpr int kMaxLevel = 21;      // 21 bits per axis, 63-bit Morton keys
constexpr int kLeafMaxLimit = 4096;
constexpr int kBboxChunk = 4096;   // bodies per bounding-box block (never across systems)

// error bits of the device error word
enum : int32_t {
    kErrNonFinite = 1,    // NaN/Inf position or mass
    kErrStack = 2,        // walk stack overflow
    kErrCapacity = 4,     // the node table outgrew its allocation
    kErrWorkLoop = 8,     // a bounded wait gave up
    kErrBand = 16,        // the learned walk's band-cell record outgrew its buffer
    kErrFmmPool = 32,     // the FMM's unresolved-source pool outgrew its allocation (regrown, rerun)
    kErrFmmSlab = 64,     // one cell's unresolved-source list outgrew its slab (regrown, rerun)
    kErrFmmStack = 128,   // the FMM's refinement stack overflowed
    kErrSortRun = 256,    // a rebuild inside a step met a run of equal top key bits too long to complete
};

// Per-system root cube (written by the bounding-box kernels).
struct SysParams {
    double c0[3];      // root cube corner
    double L;          // root cube side (power of two)
    double h;          // grid step L / 2^21
    long long qoff[3]; // c0 / h (integers): q = floor(x / h) - qoff
    int32_t qexp;      // 1 / h = 2^qexp
    float Lf;          // L as float (exact)
    float uf;          // h / 2 as float (exact): unit of the integer centres
    int32_t first;     // bodies [first, end)
    int32_t end;
    int32_t bb[6];     // bounding box as order-preserving ints: lo xyz, hi xyz
    float msys;        // total mass (for the learned correction's features)
    int32_t pad;
};

// Per-context scalars kept in device memory (written by kernels, read by
// kernels and, at synchronisation points, by the host).
struct Info {
    int32_t err;       // error bits
    int32_t depth;     // deepest level of the forest
    int64_t M;         // number of nodes
    int64_t G;         // number of groups
    int64_t cap_m;     // node table capacity (for the device-side check)
    uint32_t work[4];  // walk work-queue counters, one per launch of a force phase
    unsigned long long interactions;  // body-source interactions of the last walk
    unsigned long long cells;         // body-cell interactions (group size x accepted cells)
    unsigned long long bodies;        // body-body interactions (group size x direct-list bodies)
    double diag[8];    // KE, PE, P[3], L[3]
};

// Node record as the walk reads it (breadth-first order, index v; the roots
// of systems 0..S-1 are nodes 0..S-1).
//   a: centre of mass minus cube centre (float), mass (float)
//   b: first body, body count, first child, level | nchild << 8
//   c: cube centre in units of u = h/2 of its system (exact integers), system
//   d: centre of mass in absolute coordinates (float), mass (plain mode)
struct NodeTables {
    float4* a;
    int4* b;
    int4* c;
    float4* d;
    float* quad;     // 6 per node, second moments about the COM (FP32)
    uint4* feat;     // 2 per node: the learned correction's cell-only features (eps/s, log2 count,
                     // M / M_sys, 6 moment ratios), normalised, as BF16 pairs (words 2..7 of a row)
    double* mass64;  // the bottom-up reduction's results in FP64
    double* com64;   // 3 per node
    float4* dsum;    // 2 per node: the bottom-up sums {m, m x} as float pairs, hi parts then lo parts
};

// scratch of the radix sort / scans
struct SortBufs {
    uint64_t* keys_alt;
    uint32_t* vals_alt;
    uint32_t* ghist;                 // passes x 256 digit counts -> exclusive offsets
    unsigned long long* status;      // look-back words, passes x tiles x 256
    uint32_t* tiles;                 // tile counters, one per pass
    int32_t* err;                    // device error word (bounded look-back)
    uint32_t* blocksum;              // scan partials
    // a sort of the keys' top bits only: the starts of runs of equal top bits
    // longer than the per-thread completion takes (capacity run_cap), their count
    int64_t* runs = nullptr;
    unsigned long long* nruns = nullptr;
    int64_t run_cap = 0;
};
constexpr int kSortMaxPasses = 10;   // 8 key passes + up to 2 system passes

// ---------------------------------------------------------------- launchers
// all launches go on `s`; none synchronises.  Every launcher adds the number
// of kernels it launched to a process-wide counter (count_launches).
void count_launches(int k);
long long launches_total();
// streaming multiprocessors of the current device (cached per device; a
// host query, allowed while a stream is being captured)
int sm_count();
// records the reason of a failure outside any context (tc_last_error(NULL))
void set_thread_error(const char* msg);

// exclusive scan of n uint32 values into out (out may alias in), total to
// *total_dev (device pointer, nullable)
void scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev,
              uint32_t* blocksum, cudaStream_t s);
int64_t scan_blocksum_size(int64_t n);

// Stable LSD radix sort of (key, val) by bits [0, nbits) of key, then (if
// sys_bits > 0) by the system of each value's body, sys_of[val], so the
// result is ordered by (system, key).  Afterwards b.ghist[p * 256 + d] is
// the number of items whose pass-p digit is below d.
// low_bit > 0 (needs b.runs): the passes sort bits [low_bit, nbits) only
// (8-bit digits from low_bit up), then every run of items with equal top bits (and
// system) is put in (key, val) order by a per-run completion, so the
// result is the same as the full sort's whenever the values are distinct
// (the bodies' indices); a run longer than run_max (at most kSortRunMax)
// raises kErrSortRun and kErrCapacity instead.
constexpr int64_t kSortRunMax = 16384;
void radix_sort_u64(uint64_t* keys, uint32_t* vals, int64_t n, int nbits, const uint32_t* sys_of,
                    int sys_bits, SortBufs& b, cudaStream_t s, int low_bit = 0, int64_t run_max = kSortRunMax);
constexpr int64_t kSortRunMaxSynced = 1024;  // a synchronised build re-sorts every digit past this
constexpr int kSortMarginLevels = 2;  // levels below the last synchronised depth a step's sort orders
// The same for 32-bit keys when the item count is only known on the device:
// n_cap bounds it, *n_dev (device) holds it.
void radix_sort_u32(uint32_t* keys, uint32_t* vals, int64_t n_cap, const int64_t* n_dev, int nbits,
                    SortBufs& b, uint32_t* keys_alt32, cudaStream_t s);
int64_t radix_tiles(int64_t n);  // tiles of one pass (status words: 256 per tile per pass)
// self-test of the radix pass's bounded look-back (see tc_sort.cu)
cudaError_t sort_wait_selftest(uint64_t* keys, uint32_t* vals, uint64_t* kout, uint32_t* vout,
                               unsigned long long* status, uint32_t* counter, uint32_t* goff, int32_t* err,
                               cudaStream_t s);
int64_t sort_selftest_items();

// build pieces
void launch_sys_ids(const int64_t* offsets, int nsys, int64_t n, uint32_t* sys_of, SysParams* sysp,
                    cudaStream_t s);
void launch_bbox(const float* pos, const int4* chunks, int nchunks, SysParams* sysp, int nsys, int32_t* err,
                 cudaStream_t s);
void launch_keys(const float* pos, const float* mass, int64_t n, const uint32_t* sys_of, const SysParams* sysp,
                 uint64_t* keys, uint32_t* idx, int32_t* err, cudaStream_t s);
void launch_gather(const float* pos, const float* mass, const uint32_t* perm, int64_t n,
                   float4* body, cudaStream_t s);
void launch_node_counts(const uint64_t* keys, const uint32_t* sys_of, int64_t n, int leaf_max, int8_t* w,
                        int8_t* delta, int8_t* top, uint32_t* nstart, int32_t* depth, cudaStream_t s);
void launch_check_capacity(const uint32_t* m_total, Info* info, cudaStream_t s);
void launch_emit_preorder(const int8_t* delta, const uint32_t* nstart, const uint32_t* prepos,
                          int64_t n, const Info* info, uint32_t* pre_level, uint32_t* pre_first,
                          uint32_t* iota, cudaStream_t s);
void launch_node_finalize(const uint64_t* keys, const int8_t* top, const uint32_t* sys_of,
                          const SysParams* sysp, int64_t n, const uint32_t* bfs_level, const uint32_t* bfs_pre,
                          const uint32_t* pre_first, const uint32_t* bfs_of_pre, int64_t cap_m, const Info* info,
                          NodeTables nt, cudaStream_t s);
void launch_inverse_perm(const uint32_t* perm, int64_t cap_m, const Info* info, uint32_t* inv, cudaStream_t s);
// moments: leaves, then internal levels depth-1 .. 0 (depth < 0: the depth
// is known on the device only; with depth_hint >= 0, the depth of an earlier
// build, levels depth_hint+2 .. 0 get a launch each and any deeper ones one
// block, else all 21 levels get a launch); each level reads its range on the
// device: level_start[l] is the first node of level l (the level sort's
// digit offsets; level_start[l+1] ends it)
void launch_moments(const float4* body, int64_t cap_m, int depth, int depth_hint, const uint32_t* level_start,
                    const uint32_t* sys_of, const SysParams* sysp, const Info* info, NodeTables nt, bool quad,
                    cudaStream_t s);
void launch_group_marks(int64_t cap_m, const Info* info, const NodeTables nt, int gmax, int64_t n,
                        uint32_t* gflag, int32_t* gref_at, cudaStream_t s);
// groups by size class, stable: lists[k * cap_g + i], counts[k], class 0
// holding at most 32 bodies, class 1 at most 64, class 2 more; scratch holds
// group_split_scratch() ints
size_t group_split_scratch();
void launch_group_split(const int32_t* gfirst, const Info* info, int64_t cap_g, int32_t* lists, int32_t* counts,
                        int32_t* scratch, cudaStream_t s);
void launch_group_table(const uint32_t* gflag, const uint32_t* gscan, const int32_t* gref_at,
                        int64_t n, const uint32_t* total, int32_t* gfirst, int32_t* gref, Info* info,
                        cudaStream_t s);

// walk + force
struct WalkArgs {
    const float4* body;        // Morton order (x, y, z, m)
    const uint32_t* perm;      // Morton position -> original index
    const uint32_t* sys_of;    // body position -> system
    const SysParams* sysp;     // per-system root cube
    NodeTables nt;
    const int32_t* gfirst;     // G + 1 entries
    const int32_t* gref;       // G
    Info* info;
    float* acc;                // n x 3, original order
    float* pot;                // n, original order (nullable)
    int32_t* ncell;            // per group (nullable)
    int32_t* nbody;
    unsigned long long* hash;
    float theta2, eps2, G;
    float inv_eps;             // 1/eps for the potential self term
    // learned correction (null model: off)
    const void* mlp;           // device MlpDev
    float band2;               // accepted cells with s^2 >= band2 d^2 get a correction
    float eps;
    // training pairs (null: off): accepted cells with count >= 2 in the band
    // are emitted with probability pair_prob as (a body of the group, cell)
    int32_t* pair_body;
    int32_t* pair_node;
    unsigned long long* pair_count;
    int64_t pair_cap;
    float pair_prob;
    unsigned long long pair_seed;
    unsigned long long* mlp_evals;   // corrections evaluated (nullable)
    // list export (null: off): walk group list_group only, write its accepted
    // cells and opened leaves (walk order, at most list_cap each) and their
    // counts to list_n[0..1]; no forces or totals are written
    int32_t* list_cells;
    int32_t* list_leaves;
    int64_t list_cap;
    int64_t* list_n;
    int32_t list_group;
    // group list (null: every group 0..G-1): walk glist[0, *glist_n) only
    const int32_t* glist;
    const int32_t* glist_n;
    int work_slot;  // this launch's work-queue counter, info->work[work_slot]
    // learned correction evaluated after the walk (split walk): the band
    // cells of every group recorded as (node, group) pairs in chunks of
    // kBandChunk entries taken from *band_n (unused tails hold node -1), at
    // most band_cap entries; grec[2 g], grec[2 g + 1] the group's record for
    // the rows: {box centre in its reference cube's frame, h/2} and
    // {reference cube centre (integer units of h/2, as int bits), root side}
    int2* band;
    unsigned long long* band_n;
    int64_t band_cap;
    float4* grec;
};
constexpr int kBandChunk = 256;
struct WalkConfig {
    int gmax;         // 32, 64 or 128
    int warps;        // warps per block
    int precise;      // cell-relative sources + compensated accumulation
    int want_pot;
    int verify;
    int blocks_per_sm;
    int stack;        // walk stack entries per warp
    int tile;         // list tile entries: 64, 128 or 256
    int learned;      // 1: learned far-field correction (precise mode, no potential)
    int quadw;        // 1: accepted cells add their quadrupole term (precise mode)
    int classes;      // 1: one launch per group size class (the smaller beside the largest); 0: one launch
    int split;        // 1: monopole walks on producer/consumer warp pairs (k_walk_ws)
};
// host-side preparation of the walk kernel's launch (attributes, occupancy);
// call before a stream capture
cudaError_t prepare_walk(const WalkConfig& c, int num_sms, int* grid, size_t* smem);
// reset_totals: zero the work-queue counters and (outside list export) the
// interaction totals first -- the first launch of a force phase; the later
// launches of a phase split over size classes count on counters of their own
// (a.work_slot) zeroed with the first
cudaError_t launch_walk(const WalkArgs& a, const WalkConfig& c, int grid, size_t smem, cudaStream_t s,
                        bool reset_totals = true);

// the walk's force loop alone (tc_force_probe.cu); returns the interactions
// the launch sums
double launch_force_probe(int blocks, int reps, float* out, cudaStream_t s);

// learned far-field correction (tc_mlp.cu)
size_t mlp_dev_size();
size_t mlp_frag_size();  // the inference part at the front of a device model
size_t mlp_train_smem();
// training step on B rows: per-warp partial gradients in part (at least
// mlp_train_part_floats(blocks) floats), added in warp order into grad (the
// packed gradient, overwritten) and the loss added to *loss
int64_t mlp_train_part_floats(int blocks);
cudaError_t launch_mlp_train(const float* X, const float* T, const float* W, const int32_t* idx, int B,
                             const void* model, float* grad, float* loss, float* part, int blocks, cudaStream_t s);
void launch_mlp_pack(const float* params, const float* maps, void* model, cudaStream_t s);
void launch_adam(float* p, float* m, float* v, const float* g, int n, float lr, int t, cudaStream_t s);
void launch_mlp_infer(const float* X, int64_t n, const void* model, float* Y, cudaStream_t s);
// the learned correction evaluated after a split walk: every recorded band
// cell's row at its group's centre through the network on the tensor cores,
// F label summed per group into gcorr (G x 3, zeroed by the caller); then
// each body's acceleration gains its group's sum
void launch_band_eval(const WalkArgs& a, const void* model, float* gcorr, unsigned long long* evals,
                      cudaStream_t s);
void launch_band_apply(const Info* info, int64_t cap_g, const int32_t* gfirst, const uint32_t* perm,
                       const float* gcorr, float* acc, cudaStream_t s);
// the learned correction's per-cell features of every node for softening
// eps under the model (run before a learned walk)
void launch_node_features(const Info* info, int64_t cap_m, const SysParams* sysp, NodeTables nt, float eps,
                          const void* model, cudaStream_t s);
// the emitted (body, node) pairs sorted by (body, node): the walk emits them
// in whatever order its warps finish, the training wants one order
void launch_pair_order(int32_t* pb, int32_t* pv, int64_t np, uint64_t* keys, uint32_t* vals, SortBufs& b,
                       cudaStream_t s);
void launch_pair_labels(const int32_t* pb, const int32_t* pv, int64_t np, const float4* body, const uint32_t* sys_of,
                        const SysParams* sysp, NodeTables nt, float eps, float G, float* feat, float* lab,
                        float* fac, cudaStream_t s);
void launch_sys_mass(SysParams* sysp, int nsys, const NodeTables nt, const Info* info, cudaStream_t s);
// training data on the device: FP64 sums of x, x^2, t^2 (and F^2) over the
// pairs (kMlpSums doubles), the model's maps from them (and the factor-weight
// scale), normalised rows and scaled targets, loss weights (mode 0: check
// the given ones, mode 1: F^2 n / sum F^2; *bad = 1 for a non-finite or
// negative weight), fresh parameters, and a seeded permutation of [0, n)
constexpr int kMlpSums = 13 + 13 + 3 + 1;
void launch_mlp_sums(const float* X, const float* T, const float* F, int64_t n, double* sums, cudaStream_t s);
void launch_mlp_maps(const double* sums, int64_t n, float* maps, float* wscale, cudaStream_t s);
void launch_mlp_rows(const float* X, const float* T, int64_t n, const float* maps, float* rows, float* tout,
                     cudaStream_t s);
void launch_mlp_weights(float* w, int64_t n, int mode, const float* wscale, int32_t* bad, cudaStream_t s);
void launch_mlp_init(float* params, uint64_t seed, cudaStream_t s);
void launch_mlp_shuffle(int64_t n, uint64_t key, int32_t* idx, cudaStream_t s);

// FP32 throughput probe (8 independent FMA chains per thread, scalar or
// paired f32x2 instructions)
void launch_fp32_probe(bool paired, int blocks, int iters, float* out, cudaStream_t s);

// dynamics and diagnostics
void launch_kick_drift(float* pos, float* vel, const float* acc, int64_t n, float hkick, float dt,
                       const Info* info, cudaStream_t s);
void launch_kick(float* vel, const float* acc, int64_t n, float hkick, const Info* info, cudaStream_t s);
void launch_diag(const float* pos, const float* vel, const float* mass, const float* pot,
                 int64_t n, Info* info, cudaStream_t s);
void launch_direct(const float* pos, const float* mass, const uint32_t* sys_of, const SysParams* sysp,
                   const int64_t* idx, int64_t ns, float eps2, float G, double* acc, double* pot,
                   cudaStream_t s);

// fast multipole method (tc_fmm.cu).  Level starts: lstart[l] is the first
// breadth-first index of level l, lstart[l] = M past the deepest level
// (kFmmLevelSlots entries).  launch_fmm launches the parent table and one
// kernel per level 0..depth; its scratch: loc (cap_m x fmm_loc_width()
// floats), near_off / near_cnt (cap_m), two pools of pool_cap entries, a slab
// of slab_cap entries for each of fmm_slab_warps() warps, ctr (8 counters:
// pool fill per level parity, pool need, slab need, M2L pairs, P2P pairs and
// their two hashes; zero the last six before the launch); rec: per node its
// M2L and P2P pairs as target and their hashes.
constexpr int kFmmLevelSlots = kMaxLevel + 3;
struct FmmLaunch {
    const float4* body;
    const uint32_t* perm;
    const SysParams* sysp;
    NodeTables nt;
    const Info* info;
    int32_t* err;
    int64_t cap_m;
    int32_t* parent;
    float* loc;
    int32_t* pool[2];
    int64_t pool_cap;
    int32_t* slab;
    int64_t slab_cap;
    int64_t* near_off;
    int32_t* near_cnt;
    unsigned long long* ctr;
    unsigned long long* rec;  // 4 per node (M2L pairs, P2P pairs, their hashes), 32-byte aligned
    double* rad;              // per node: r_X (FP64)
    int4* fnode;              // per node, 3 entries: the walk's record with r_X in FP32
    int records;              // pair-set hashes and per-node records (else counts only)
    float* acc;
    float theta, eps, G;
};
int64_t fmm_slab_warps();
int fmm_loc_width();
void launch_fmm_level_starts(const Info* info, int64_t cap_m, NodeTables nt, int64_t* lstart, cudaStream_t s);
cudaError_t launch_fmm(const FmmLaunch& p, const int64_t* lstart_h, int depth, cudaStream_t s);

}  // namespace tc
