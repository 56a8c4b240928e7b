/*
 * tc_oracle.h -- plain, slow FP64 CPU oracle of the treecode force phase.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
 * and its Python binding) may include, link or call this code; only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark do.  It
 * shares no source, header, table or helper with the GPU path.
 *
 * What it computes follows the paper's treecode (Sec. 3.1):
 *   - the space is divided recursively into 8 sub-cubes until a cube holds
 *     no more than a threshold of bodies (the oct-tree),
 *   - each cell carries its total mass and centre of mass,
 *   - the force on a body is found by walking the tree from the root: a
 *     cell far enough away joins the interaction list, otherwise the walk
 *     descends into its children; the list is then summed with the
 *     gravitational force law F = G m_a m_b / r^2 (Sec. 3.1 equation),
 *   - bodies then update position and velocity (Sec. 3.1, last paragraph).
 * Readings of what the paper leaves open (root cube, Morton keys, groups,
 * opening test, softening, integrator) are stated at each function.
 *
 * All arithmetic is IEEE double, compiled with -ffp-contract=off.
 */
#ifndef TC_ORACLE_H
#define TC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAX_LEVEL 21 /* 21 bits per axis, 63-bit keys */

typedef struct or_tree or_tree;

/* Root cube: out[0..2] = corner c0, out[3] = side L, out[4] = grid step
 * h = L / 2^21.  Returns 0, or -1 for n < 1 or a non-finite coordinate. */
int or_root_cube(const float *pos, int64_t n, double *out5);

/* Morton keys of n bodies for a given root cube (out of or_root_cube). */
void or_keys(const float *pos, int64_t n, const double *cube5, uint64_t *keys);

/* Build the oct-tree of n bodies (pos n x 3, mass n) with leaf threshold
 * leaf_max.  Returns NULL on invalid input (n < 1, leaf_max < 1, NaN/Inf,
 * a mass that is not positive). */
or_tree *or_tree_build(const float *pos, const float *mass, int64_t n, int leaf_max);
void or_tree_free(or_tree *t);

int64_t or_tree_nnodes(const or_tree *t);
int64_t or_tree_nbodies(const or_tree *t);
void or_tree_get_cube(const or_tree *t, double *out5);
/* perm[k] = original index of the body at sorted (Morton) position k. */
void or_tree_get_perm(const or_tree *t, uint32_t *perm);
void or_tree_get_keys(const or_tree *t, uint64_t *keys_sorted);
/* Node table in breadth-first order (by level, then by first body). */
void or_tree_get_nodes(const or_tree *t, int32_t *level, uint64_t *prefix,
                       int64_t *first, int64_t *count, int64_t *child_first,
                       int32_t *nchild, int64_t *parent);
/* mass[M], com[M*3] (absolute), quad[M*6] = Qxx,Qxy,Qxz,Qyy,Qyz,Qzz. */
void or_tree_get_moments(const or_tree *t, double *mass, double *com, double *quad);

/* Body groups for the group walk; returns the number of groups G. */
int64_t or_tree_make_groups(or_tree *t, int gmax);
void or_tree_get_groups(const or_tree *t, int64_t *first, int64_t *count, int64_t *ref);

/* Walk + force for groups [g_begin, g_end).
 *   acc, pot : n x 3 / n, ORIGINAL body order; only bodies of the walked
 *              groups are written.  pot may be NULL.
 *   amag  : n, ORIGINAL order, sum over the list of |term| (the scale of the
 *           rounding error of the sum); may be NULL.
 *   ncell, nbody : per group (indexed by group id, length G), list lengths.
 *   hash  : per group order-independent hash of the accepted cells and the
 *           opened leaves.
 *   flag  : per group 1 if any opening test it evaluated lay within the
 *           1e-6 relative tie band, else 0.
 * Any of ncell, nbody, hash, flag may be NULL.
 * Returns the number of body-source interactions evaluated. */
int64_t or_tree_walk(const or_tree *t, double theta, double eps, double G,
                     int64_t g_begin, int64_t g_end, double *acc, double *pot, double *amag,
                     int64_t *ncell, int64_t *nbody, uint64_t *hash, int32_t *flag);

/* The same walk with, for quadrupole != 0, every accepted cell's quadrupole
 * term added to its monopole: with d = com - x, rho^2 = |d|^2 + eps^2 and Q
 * the cell's second moments about its centre of mass (second-order Taylor
 * expansion of the softened potential),
 *   phi_Q = -(G/2) (3 d.Qd / rho^5 - tr Q / rho^3)
 *   a_Q   = G (-3 Qd / rho^5 + (7.5 d.Qd / rho^7 - 1.5 tr Q / rho^5) d).
 * amag then also sums |a_Q| per component. */
int64_t or_tree_walk_order(const or_tree *t, double theta, double eps, double G, int quadrupole,
                           int64_t g_begin, int64_t g_end, double *acc, double *pot, double *amag,
                           int64_t *ncell, int64_t *nbody, uint64_t *hash, int32_t *flag);

/* The interaction list of group g at theta: accepted cells and opened
 * leaves (node indices) in the walk's order; at most cap_c / cap_l written,
 * *nc / *nl = the full lengths. */
void or_tree_group_list(const or_tree *t, double theta, int64_t g, int64_t *cells, int64_t cap_c,
                        int64_t *leaves, int64_t cap_l, int64_t *nc, int64_t *nl);

/* For tests: the opening-test decision of one (group, node) pair:
 * 0 = open (contains a group body), 1 = open (too close), 2 = accept. */
int or_tree_test(const or_tree *t, int64_t group, int64_t node, double theta);

/* Direct O(N*S) sum for the bodies idx[0..ns) (ORIGINAL indices) over all n
 * bodies; acc is ns x 3, pot (nullable) ns.  Float and double inputs. */
void or_direct(const float *pos, const float *mass, int64_t n, double eps, double G,
               const int64_t *idx, int64_t ns, double *acc, double *pot);
void or_direct64(const double *pos, const double *mass, int64_t n, double eps, double G,
                 const int64_t *idx, int64_t ns, double *acc, double *pot);

/* Leapfrog pieces (kick-drift-kick), in place, double precision. */
void or_kick(double *vel, const double *acc, int64_t n, double h);
void or_drift(double *pos, const double *vel, int64_t n, double dt);

/* out[0] = kinetic energy, out[1] = potential energy 0.5*sum m*pot,
 * out[2..4] = linear momentum, out[5..7] = angular momentum. */
void or_diag(const double *pos, const double *vel, const double *mass,
             const double *pot, int64_t n, double *out8);

/* ---- Learned far-field correction (a growth of the method; no paper
 * counterpart).  For a point x and a cell v (side s, mass M, centre of mass
 * c, second moments Q about c, count bodies), with d = c - x and r = |d|:
 *   features (13): d/s (3), s/r, eps/s, log2(count), M/msys, Q_ab/(M s^2)
 *                  in the order xx, xy, xz, yy, yz, zz (6)
 *   factor:        G M s^2 / r^4, the scale of the quadrupole term
 *   label (3):     (a_exact - a_mono) / factor, where a_exact is the
 *                  softened direct sum over the cell's bodies and a_mono the
 *                  softened monopole G M d / (r^2 + eps^2)^(3/2).          */
void or_mlp_features(const or_tree *t, int64_t node, const double *x, double eps, double msys, double *f13);
double or_mlp_factor(const or_tree *t, int64_t node, const double *x, double G);
void or_mlp_label(const or_tree *t, int64_t node, const double *x, double eps, double G, double *t3);

/* MLP 13 -> 64 -> 64 -> 3 with ReLU after the hidden layers.  Parameters
 * packed: W1[13][64], b1[64], W2[64][64], b2[64], W3[64][3], b3[3]
 * (W[i][j] couples input i to output j), OR_MLP_NPARAM values. */
#define OR_MLP_NPARAM (13 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3)
void or_mlp_forward(const double *params, const double *X, int64_t n, double *Y);
/* loss L = (1/n) sum_i w_i |Y_i - T_i|^2 (w NULL: all 1) and its gradient
 * (packed like params) */
double or_mlp_grad(const double *params, const double *X, const double *T, const double *w, int64_t n,
                   double *grad);

/* BF16 rounding model of the network: the normalised inputs, the weights
 * and the hidden activations after the ReLU rounded to bfloat16 (nearest,
 * ties to even), sums exact; in the backward pass the operands of the
 * gradient products (dY, dH2, dH1) rounded too, the bias gradients from the
 * unrounded values.  R / grad_rad / loss_rad (nullable) get the radius
 * around each model value within which an implementation performing the
 * same roundings on FP32 sums must land, given inputs within Xr (nullable:
 * exact) of X before their rounding. */
double or_bf16(double x);
void or_mlp_forward_bf16(const double *params, const double *X, const double *Xr, int64_t n, double *Y,
                         double *R);
double or_mlp_grad_bf16(const double *params, const double *X, const double *Xr, const double *T,
                        const double *w, int64_t n, double *grad, double *grad_rad, double *loss_rad);

/* Learned correction of the group walk for groups [g_begin, g_end): every
 * accepted cell of a group's walk with two or more bodies and s >= band * d
 * (d = distance from its centre of mass to the group's box) is evaluated at
 * the centre x_g of the group's box; factor(x_g) y (factor G M s^2 / r^4,
 * r = |com - x_g|) is added to corr (n x 3, ORIGINAL order) for every body of the group.
 *   y = network((f - maps[0..12]) * maps[13..25]) * maps[26..28]
 * or, with params NULL, the exact label at x_g.  flag[g] (nullable) = 1 when
 * an opening or band test of the group lay within 1e-6 relative of its
 * bound.  Returns the number of cell evaluations. */
int64_t or_tree_learned(const or_tree *t, double theta, double eps, double G, double band,
                        const double *params, const double *maps, int64_t g_begin, int64_t g_end,
                        double *corr, int32_t *flag);
/* The same band sum with the network's BF16 rounding model (or_mlp_forward_bf16;
 * params required): crad (n x 3) gets the radius within which an FP32
 * implementation lands -- its features computed in FP32 at the same point
 * (radii from an error analysis of that evaluation), normalised, run
 * through the rounding model, scaled by factors computed in FP32 and summed
 * over the group's cells in FP32. */
int64_t or_tree_learned_bf16(const or_tree *t, double theta, double eps, double G, double band,
                             const double *params, const double *maps, int64_t g_begin, int64_t g_end,
                             double *corr, double *crad, int32_t *flag);

/* Fast multipole method on the same tree (a reading of Sec. 5, stated in
 * tc_oracle.c): monopoles at the cells' centres of mass, third-order local
 * expansions, pair acceptance r_A + r_B < theta |c_A - c_B| (r_X: the
 * cell's radius about its centre of mass, or_fmm_radii), dual traversal,
 * M2L / L2L / L2P and P2P between leaves.  acc (n x 3, original order);
 * stats (nullable, 5): M2L pairs, P2P pairs, ties, M2L and P2P pair-set
 * hashes. */
void or_fmm(const or_tree *t, double theta, double eps, double G, double *acc, int64_t *stats);
/* r_X (M): a leaf's farthest body from its centre of mass; above, the
 * farthest child sphere, max over children (|c_child - c_X| + r_child). */
void or_fmm_radii(const or_tree *t, double *rad);
/* The same with per-target-cell records (each nullable, M entries): M2L and
 * P2P pairs whose target is the cell, their pair-set hashes, and a flag set
 * when the cell or one of its ancestors tested a pair within 1e-6 relative
 * of the acceptance bound (a decision that rounding may flip, and with it
 * every pair its subtree is handed). */
void or_fmm_nodes(const or_tree *t, double theta, double eps, double G, double *acc, int64_t *stats,
                  int64_t *nm2l, int64_t *np2p, uint64_t *hm2l, uint64_t *hp2p, int32_t *flag);

#ifdef __cplusplus
}
#endif
#endif
