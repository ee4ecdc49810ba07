/*
 * bh.h -- C ABI of libbh.so: group-shared Barnes-Hut tree force evaluation
 * on one GB300 (sm_103a), after Iwasawa et al., "Implementation and
 * performance of Barnes-Hut N-body algorithm on extreme-scale heterogeneous
 * many-core architectures" (arXiv:1907.02289).
 *
 * The path (Sec. 4.2, steps 3a-3d and 4): Morton keys, radix sort, octree,
 * node moments, groups, one tree walk per group that emits its interaction
 * list, the force kernel that sums Eq. (1) over the list particles and the
 * centre-of-mass (+ quadrupole) term over the list cells, and the leapfrog
 * update, with lists reused for several steps (the persistent interaction
 * list of Sec. 4.2) and an FP32 kernel on coordinates shifted to a group
 * origin (Sec. 4.7).
 *
 * Conventions
 *  - Every function returns an int status (BH_OK = 0 or a BH_E_* code) and
 *    never aborts; bh_last_error() gives a message for the last failure.
 *  - Particle arrays are CALLER-OWNED DEVICE memory, structure of arrays:
 *    x,y,z,vx,vy,vz,m (double) and id (int64), each of length n, plus the
 *    outputs ax,ay,az (double).  A list-constructing call permutes x..id in
 *    place into key order; id keeps particle identity.
 *  - Tree, list and scratch buffers are LIBRARY-OWNED device memory inside
 *    the context; they are allocated with cudaMalloc and grown on demand.
 *  - Work is issued on the CUDA stream given to bh_create.  Calls that must
 *    size buffers (building trees and lists) synchronise that stream; force
 *    and step calls do not, except where stated.  Device-side error words are
 *    checked at the next synchronising call (or bh_sync).
 *  - bh_get_* read-back functions copy into CALLER-OWNED HOST buffers sized
 *    from bh_get_sizes, and synchronise the stream.
 *  - A context is used by one host thread at a time (calls on one context
 *    are not synchronised against each other); separate contexts are
 *    independent.  Make every call with the device current that was
 *    current at bh_create (the context's buffers live there).
 */
#ifndef BH_H
#define BH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BH_OK 0
#define BH_E_INVAL 1         /* bad parameter, size or non-finite position   */
#define BH_E_NOMEM 2         /* device allocation failed                     */
#define BH_E_CUDA 3          /* a CUDA call failed                           */
#define BH_E_LIST_OVERFLOW 4 /* list or node buffer too small (needed size   */
                             /* is reported by bh_get_sizes)                 */
#define BH_E_TIMEOUT 5       /* reserved: no kernel of this library waits on */
                             /* the device (no spin on a flag, a barrier or  */
                             /* another kernel), so it is never returned     */
#define BH_E_STATE 6         /* call out of order (e.g. forces before lists) */

#define BH_PREC_FP64 0 /* plain FP64 force kernel                              */
#define BH_PREC_FP32 1 /* FP32 kernel, coordinates relative to a group origin */

/* bh_compute_forces flags */
#define BH_FORCE_TREE_ONLY 1 /* do not add the central-mass term */

typedef struct bh_ctx bh_ctx;

/* Method parameters (paper symbols where it has them).
 *  theta      opening angle (>= 0); the paper names no criterion, this
 *             library opens a node when side > theta * box gap (integer
 *             boxes on the key grid, conservative), or when the gap is
 *             within r_coll.
 *  eps        Plummer softening added to gravity (0 for rings).
 *  G          gravitational constant (1 in the paper).
 *  M_central  central mass at the origin (the planet, Table 1); 0 = none.
 *  r_coll, kappa, eta   contact distance and spring/dashpot constants of
 *             Eq. (1) (the paper fixes only restitution 0.5).
 *  dt         leapfrog step.
 *  n_g        largest group (groups are the maximal tree nodes holding at
 *             most n_g particles, Sec. 4.2).
 *  n_leaf     largest leaf (1 <= n_leaf <= n_g).
 *  order      1 = centre of mass only (Sec. 5.1), 2 = plus quadrupole.
 *  precision  BH_PREC_FP64 or BH_PREC_FP32 (Sec. 4.7).
 *  rebuild_every  force evaluation k rebuilds keys..lists iff
 *             k % rebuild_every == 0, otherwise refreshes moments only.
 *  key_frame  frame of the keys, the tree and the opening test (forces are
 *             always Cartesian): 0 = (x, y, z); 1 = cylindrical (phi, r, z),
 *             Sec. 4.3, for a narrow ring about the z axis near r ~ 1, where
 *             those coordinates measure distance like Cartesian ones.  phi is
 *             periodic in the opening test, and the contact clause uses
 *             r_coll / r_min (r_min: the smallest particle radius of the
 *             patch), so no contact pair is missed.  Needs r > 0 for every
 *             particle (BH_E_INVAL otherwise, at the list build).
 *  list_capacity  most interaction-list entries one list build may hold:
 *             particle-list entries (opened leaves) + cell-list entries
 *             (accepted nodes) + list particles (the leaves' particles, the
 *             form the force kernels read); 0 = no limit (buffers grow on
 *             demand).  A build that needs more fails with
 *             BH_E_LIST_OVERFLOW before writing any list; bh_get_sizes then
 *             reports the sizes it needs, and bh_set_list_capacity changes
 *             the limit.
 *  omega      rotation rate of the frame the particle arrays are kept in
 *             (Sec. 4.4: coordinates rotating at the Kepler rate of the ring
 *             centre, so that particles there barely move): 0 = inertial.
 *             With omega != 0 every step's drift is followed by the rotation
 *             of x, y and vx, vy by -omega dt about the z axis (x' = c x + s y,
 *             y' = -s x + c y, c = cos(omega dt), s = sin(omega dt)), so the
 *             arrays hold positions and inertial velocities in axes that turn
 *             with the frame; keys, trees and lists are built there.  The
 *             forces are rotation-invariant (the central mass sits on the axis),
 *             so this is the inertial integration seen from the turning axes. */
typedef struct {
    double theta, eps, G, M_central, r_coll, kappa, eta, dt;
    int n_g, n_leaf, order, precision;
    int rebuild_every, key_frame;
    int64_t list_capacity;
    double omega;
} bh_params;

/* Caller-owned device arrays (see Conventions). */
typedef struct {
    double *x, *y, *z, *vx, *vy, *vz, *m;
    int64_t* id;
    double *ax, *ay, *az;
    int64_t n;
} bh_particles;

/* Stages of the path timed by bh_set_timing (indices of bh_counters.stage_ms):
 *  KEYS      cylindrical coordinates (key_frame 1), root box, Morton keys   (a1)
 *  SORT      stable radix sort of (key, index)                              (a2)
 *  PERMUTE   gather of the particle arrays into key order                   (a2)
 *  TREE      octree levels, integer node boxes and walk records             (a3)
 *  MOMENTS   node moments (every evaluation)                                (a4)
 *  GROUPS    groups                                                         (a5)
 *  LISTS     tree walk, list expansion and the FP32 kernel's group order (a6, a7)
 *  SPLIT     FP32 path: hi/lo split of the particles (every evaluation)
 *  FORCE     force kernel                                                   (a8)
 *  CONTACTS  FP32 path: the FP64 contact pass after the force kernel        (a8)
 *  UPDATE    leapfrog kicks and drift                                       (a9)
 *  REFINE    FP32 path: re-evaluation of ill-conditioned particles         (a8) */
#define BH_STAGE_KEYS 0
#define BH_STAGE_SORT 1
#define BH_STAGE_PERMUTE 2
#define BH_STAGE_TREE 3
#define BH_STAGE_MOMENTS 4
#define BH_STAGE_GROUPS 5
#define BH_STAGE_LISTS 6
#define BH_STAGE_SPLIT 7
#define BH_STAGE_FORCE 8
#define BH_STAGE_CONTACTS 9
#define BH_STAGE_UPDATE 10
#define BH_STAGE_REFINE 11
#define BH_N_STAGES 12

/* Interaction and timing counters of the last force evaluation. */
typedef struct {
    int64_t n_groups;
    int64_t n_pp; /* particle-particle interactions (i, list particle) incl. i = j */
    int64_t n_pc; /* particle-cell interactions                                   */
    int64_t n_evals;    /* force evaluations since the last list build            */
    int64_t n_rebuilds; /* list-constructing evaluations so far                   */
    int64_t n_launches; /* CUDA kernels launched by this context                  */
    int64_t n_contacts; /* contact candidates of the last FP32 force evaluation   */
    int64_t n_pp_far;   /* FP32 path: the part of n_pp whose list particle is "far"
                         * (beyond contact reach and at least an eighth of the
                         * group's largest side away), evaluated with a single
                         * FP32 separation relative to the group origin; 0 on
                         * the FP64 path                                       */
    int64_t n_one_walk_builds; /* list builds whose lists came from a single tree
                         * walk into per-group slots (sized from the previous
                         * build's longest lists) instead of a count walk and a
                         * fill walk; results are the same either way          */
    int64_t n_h2d_bytes; /* bytes bh_step_host has copied host -> device so far  */
    int64_t n_d2h_bytes; /* ... and device -> host (ids, and masses on the way
                          * back, only for calls with a list-constructing
                          * evaluation: other steps leave them unchanged)        */
    int64_t n_refined;   /* FP32 path: particles of the last force evaluation whose
                          * FP32 sum was ill-conditioned, |a_i| < 0.12 G x the
                          * root of the sum of the squares of its FP32 tile
                          * partial sums (a particle whose neighbours' pulls
                          * nearly cancel), and which the refinement pass
                          * evaluated again over the same lists in df (pairs
                          * of FP32 numbers) arithmetic; 0 on the FP64 path    */
    double stage_ms[BH_N_STAGES];     /* device time of each stage (CUDA events on the
                                       * context's stream) summed over the calls made
                                       * with timing on since the last reset
                                       * (bh_get_timing); the stages of steps run
                                       * as a graph are not timed                */
    int64_t stage_calls[BH_N_STAGES]; /* timed calls of each stage                */
    int64_t n_graph_builds;      /* list-constructing steps of bh_step run as one CUDA
                                  * graph launch (bh_tuning.graph = 1)          */
    int64_t n_graph_build_redos; /* ... of those, steps whose buffers (sized from the
                                  * previous build with room to grow) turned out
                                  * too small: the graph stopped after the reordering
                                  * and the step was finished eagerly, with the
                                  * same result                                 */
    int64_t n_graph_captures;    /* step graphs captured (and instantiated) so far,
                                  * list-reusing and list-constructing         */
} bh_counters;

/* Create a context.  stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: BH_E_INVAL for theta < 0, n_g < 1, n_leaf < 1, n_leaf > n_g,
 * order not 1/2, precision not 0/1, rebuild_every < 1, key_frame not 0/1,
 * dt < 0. */
int bh_create(const bh_params* p, void* stream, bh_ctx** out);

/* Create a context for n_patches INDEPENDENT particle sets ("patches", e.g.
 * separate ring sectors) that are stepped together: the particle arrays hold
 * the patches one after another, patch q being [offsets[q], offsets[q+1]).
 * Each patch gets its own root box, keys, sort, tree, groups and lists
 * exactly as if it were alone (a patch never interacts with another), but
 * every stage runs once over all patches: one sort, one tree pass per level,
 * one walk, one force launch.  Trees form a forest whose roots are nodes
 * 0..n_patches-1; node, group and list ids are global.  offsets is a host
 * array of n_patches + 1 entries (copied): offsets[0] = 0, strictly
 * increasing, offsets[n_patches] = the n passed later (< 2^31).
 * Errors: as bh_create, plus BH_E_INVAL for n_patches outside 1..65535 or bad
 * offsets.
 * n_patches = 1 is bh_create. */
int bh_batch_create(const bh_params* p, int n_patches, const int64_t* offsets, void* stream, bh_ctx** out);
int bh_destroy(bh_ctx* ctx);
const char* bh_last_error(const bh_ctx* ctx);
int bh_set_stream(bh_ctx* ctx, void* stream);

/* Sec. 4.2 step 3a (list-constructing step): root box and Morton keys,
 * stable radix sort, in-place permutation of the particle arrays into key
 * order, level-by-level octree (BFS numbering), integer node boxes, node
 * moments and groups.  Synchronises.  Errors: BH_E_INVAL for n < 1 or
 * n >= 2^31 or a non-finite coordinate. */
int bh_build_tree(bh_ctx* ctx, bh_particles* p);

/* Sec. 4.2 step 3d, first half: one depth-first walk per group builds its
 * particle list (opened leaves) and cell list (accepted nodes), both in
 * order of first particle, and the list-reuse schedule starts.
 * Synchronises.  BH_E_STATE without a tree. */
int bh_make_lists(bh_ctx* ctx);

/* Sec. 4.2 step 3d, second half (and the list-reusing step): refresh node
 * moments from the current positions (same tree, groups and lists), then
 * the force kernel writes ax,ay,az = sum over list particles of Eq. (1)
 * + sum over list cells of the multipole term, plus the central-mass term
 * unless flags has BH_FORCE_TREE_ONLY.  Particles must be in the order of
 * the last bh_build_tree.  Asynchronous.  BH_E_STATE without lists. */
int bh_compute_forces(bh_ctx* ctx, bh_particles* p, int flags);

/* Sec. 4.2 step 4 with list reuse: nsteps kick-drift-kick leapfrog steps.
 * Force evaluation k (counted over the context's life, k = 0 the first)
 * rebuilds tree and lists iff k % rebuild_every == 0, otherwise reuses them.
 * The first call evaluates the initial acceleration.  On return the arrays
 * hold positions/velocities at the full step and ax..az the total
 * acceleration there.  Synchronises on list-constructing steps. */
int bh_step(bh_ctx* ctx, bh_particles* p, int nsteps);

/* Same as bh_step with HOST particle arrays: each call copies the arrays to
 * library-owned device buffers, steps, and copies x..id and ax..az back.
 * Only list-constructing evaluations reorder the particles, so a call with
 * none of them copies neither ids (either way) nor masses (back): they are
 * unchanged and the host arrays stay current; a later list-constructing
 * call copies the host ids in before reordering them.  Positions, masses
 * and ids are copied back on a second stream while the last evaluation's
 * force kernel runs.  Synchronises. */
int bh_step_host(bh_ctx* ctx, bh_particles* host, int nsteps);

/* Wait for the stream and report device-side errors. */
int bh_sync(bh_ctx* ctx);

/* Sizes of the current structures (any pointer may be NULL).  After a list
 * build that failed with BH_E_LIST_OVERFLOW the three list sizes are the ones
 * that build needed (their sum is the capacity it asked for). */
int bh_get_sizes(bh_ctx* ctx, int64_t* n_nodes, int64_t* n_groups, int64_t* n_pp_entries,
                 int64_t* n_pc_entries, int64_t* n_list_particles);

/* Read-backs into host buffers (n, n_nodes, n_groups, ... entries).
 * bh_get_keys: the sorted keys and perm[i] = index, before the last sort, of
 * the particle now at i.  bh_get_root writes one box per patch: lo3[3 q + a],
 * L[q] (in (phi, r, z) for the cylindrical frame).  bh_get_moments: M[node],
 * centre of mass c3[a * n_nodes + node], traceless quadrupole
 * Q6[6 node + {xx, yy, zz, xy, xz, yz}]; on the FP64 path the FP64 moments,
 * on the FP32 path the FP32 records widened to FP64 (centre = hi + lo).  bh_get_lists: CSR offsets (n_groups + 1) and
 * node ids, particle list = opened leaves, cell list = accepted nodes. */
int bh_get_keys(bh_ctx* ctx, uint64_t* keys, uint32_t* perm);
int bh_get_root(bh_ctx* ctx, double* lo3, double* L);
int bh_get_tree(bh_ctx* ctx, uint8_t* level, uint32_t* begin, uint32_t* end, int32_t* parent,
                int32_t* first_child, uint8_t* nchild, uint32_t* qlo3, uint32_t* qhi3);
int bh_get_moments(bh_ctx* ctx, double* M, double* c3, double* Q6);
int bh_get_groups(bh_ctx* ctx, int32_t* group_nodes);
int bh_get_lists(bh_ctx* ctx, int64_t* pp_off, int32_t* pp_ids, int64_t* pc_off, int32_t* pc_ids);
/* Counters; when timing is on this synchronises the stream to read the
 * stage events. */
int bh_get_counters(bh_ctx* ctx, bh_counters* out);

/* Change list_capacity (see bh_params) for later list builds; entries >= 0.
 * Errors: BH_E_INVAL for entries < 0. */
int bh_set_list_capacity(bh_ctx* ctx, int64_t entries);

/* Measurement hooks.  bh_set_timing(ctx, 1) makes every force-kernel launch,
 * and every stage of the path (BH_STAGE_*), record a pair of CUDA events on
 * the context's stream.  In a step issued as a CUDA graph only the force
 * kernel is timed (event-record nodes around it, given a fresh pair of
 * events at each launch); its other stages are not;
 * bh_get_timing synchronises the stream and returns the summed force-kernel
 * time (ms) and the number of timed launches, clearing them and the stage
 * times of bh_counters when reset != 0. */
int bh_set_timing(bh_ctx* ctx, int enable);
int bh_get_timing(bh_ctx* ctx, double* force_ms, int64_t* force_launches, int reset);

/* Launch tuning (the persistent-kernel schedule of Sec. 4.6's load balance,
 * and the knobs the autotuner searches).  Schedules of the FP32 force kernel:
 *  BH_SCHED_GRID     one warp per group, grid sized to the groups;
 *  BH_SCHED_STATIC   persistent grid (as many blocks as fit on the GPU), each
 *                    warp takes every (warps in grid)-th group of the order;
 *  BH_SCHED_DYNAMIC  persistent grid, each warp draws its next group from an
 *                    atomic ticket counter (dynamic longest-first when
 *                    order_by_cost is set).
 * Groups are taken in order of size class, and, with order_by_cost, by
 * decreasing estimated cost n_i (n_i + list particles + 2 list cells) within
 * a class. */
#define BH_SCHED_GRID 0
#define BH_SCHED_STATIC 1
#define BH_SCHED_DYNAMIC 2
typedef struct {
    int n_g;           /* group size limit; a change forces a list build at the next evaluation */
    int chunk;         /* particles of a group per warp pass: 32, 64 or 96 */
    int warps;         /* warps per block of the FP32 force kernel, 1..8 */
    int sched;         /* BH_SCHED_* */
    int order_by_cost; /* 0 or 1 */
    int graph;         /* 1: bh_step issues every step as one CUDA graph launch.
                          A list-reusing step (kick-drift, moment refresh,
                          force kernel, contact pass, kick) is captured after
                          each list build.  A list-constructing step (kick-
                          drift, keys, sort, reordering, tree, moments,
                          groups, walk, lists, forces, kick) reads no size
                          back while it runs: its buffers are sized from the
                          previous build with graph_room percent to grow and
                          it is captured again when a build has used half of
                          that room; a step that outgrows them stops after the
                          reordering and is finished eagerly (same result;
                          bh_counters.n_graph_build_redos).  The step waits
                          once, at its end, for the new list sizes.  A list
                          capacity (bh_params.list_capacity) keeps list-
                          constructing steps eager.  2: list-reusing steps
                          only.  In graph steps the contact pass reads its
                          count on the device, and an overflow of its buffer
                          is reported (BH_E_LIST_OVERFLOW) at the next
                          synchronising call */
    int order_window;  /* 0: one global size-class order; w > 0: the size-class
                          order is applied within windows of w consecutive
                          groups (list order = Morton order), so the warps in
                          flight work on nearby groups whose list data share L2 */
    int graph_contact_room; /* contact candidates a graph step may hold: 0 = twice
                          the last eager evaluation's count + 65536; n > 0 = n.
                          More candidates than that in a graph step are
                          dropped and reported as BH_E_LIST_OVERFLOW at the
                          next synchronising call (that step's contact terms
                          are then incomplete); eager evaluations always grow
                          the buffer instead */
    int graph_room;    /* list-constructing graph steps: percent of room over the
                          last build's node, group and list counts that their
                          buffers get (0..1000, default 25) */
} bh_tuning;
/* Errors: BH_E_INVAL for a value out of range (n_g < n_leaf included). */
int bh_set_tuning(bh_ctx* ctx, const bh_tuning* t);
int bh_get_tuning(bh_ctx* ctx, bh_tuning* t);

/* Autotuner: times candidate settings on the caller's particles and keeps
 * the fastest.  First the launch settings on the current n_g by force-kernel
 * time, one knob at a time (schedule, then warps in {2, 4, 8}, chunk in
 * {32, 64, 96}, order_window in {0, 2048, 8192}); then n_g in
 * {64, 96, 128, 192, 256} (those >= n_leaf) by the cost of one step, force
 * time plus list-build time / rebuild_every; then every pair of chunk and
 * order_window on the chosen n_g.  Each candidate keeps the best of three timed
 * evaluations, after untimed ones following each list build.  Like a list build it reorders the particle arrays; on
 * return the lists are built with the chosen settings, ax..az hold the
 * acceleration at the current positions, and the list-reuse schedule starts
 * afresh.  best_ms (may be NULL) receives the chosen setting's step cost.
 * Synchronises.  graph is left as set. */
int bh_autotune(bh_ctx* ctx, bh_particles* p, double* best_ms);

/* Diagnostics of the current state (the energy, momentum and collision
 * statistics a ring simulation reports alongside its steps).  Sums over all
 * particles of p (all patches), in FP64 with a fixed reduction order, so
 * repeated calls on the same state give identical bits:
 *   mass = sum m;  momentum = sum m v;  angular_momentum = sum m x cross v
 *   (about the origin);  kinetic = sum m |v|^2 / 2;  potential_central =
 *   -sum G M_central m / |x|.
 * Self-gravity potential energy is not computed (the force kernels produce
 * accelerations only).  Contact statistics of the last FP32 force evaluation
 * (-1 on the FP64 path or without contacts, whose kernel evaluates contacts
 * inline): contact_candidates = (i, j) pairs that went to the FP64 contact
 * pass, contacts = unordered pairs found with r <= r_coll.  Synchronises. */
typedef struct {
    double mass, momentum[3], angular_momentum[3], kinetic, potential_central;
    int64_t contact_candidates, contacts;
} bh_diagnostics;
int bh_get_diagnostics(bh_ctx* ctx, const bh_particles* p, bh_diagnostics* out);

/* Self-gravity potential over the current lists (the energy the ring's
 * diagnostics need besides bh_get_diagnostics' kinetic and central terms;
 * Sec. 5.1 times steps with their diagnostics), in FP64 whatever the
 * precision: node moments are recomputed in FP64 from the current positions,
 * then for every particle phi_i = sum over its group's own particles and list
 * particles (j != i) of the potential of Eq. (1)'s gravity,
 *   -G m_j / sqrt(r^2 + eps^2) for r > r_coll, and inside r_coll (where the
 *   gravity is held at its r_coll value) -G m_j / s - G m_j (r_coll^2 - r^2)
 *   / (2 s^3), s^2 = r_coll^2 + eps^2 (continuous at r_coll),
 * plus over its list cells -G M / R - G/2 R.Q.R / R^5 (R = x_i - centre,
 * R^2 including eps^2; quadrupole term for order 2).
 *  phi  [n] caller-owned device array for phi_i, or NULL.
 *  W    host double for W = 1/2 sum m_i phi_i (fixed-order FP64 reduction,
 *       bit-reproducible), or NULL; when given, the call synchronises.
 * Particles must be in the order of the last list build.  The contact
 * spring and dashpot have no potential here.  BH_E_STATE without lists. */
int bh_compute_potential(bh_ctx* ctx, const bh_particles* p, double* phi, double* W);

/* Load balance of the last persistent force launch made with timing on
 * (bh_set_timing): busy fraction = sum over warps of (finish - start) /
 * (warps x (last finish - first start)).  BH_E_STATE if there is none. */
int bh_get_balance(bh_ctx* ctx, double* busy_fraction);

/* Peak arithmetic rate of this device, measured: a kernel of independent
 * fused multiply-add chains on every SM (FP32 for kind BH_PEAK_FP32, FP64 for
 * BH_PEAK_FP64), timed with CUDA events after a warm-up launch (2 flops per
 * FMA).  Runs on the legacy default stream of the current device and
 * synchronises.  Allocates a small output buffer (freed before returning).
 * Errors: BH_E_INVAL for an unknown kind or NULL tflops, BH_E_CUDA. */
#define BH_PEAK_FP32 0
#define BH_PEAK_FP64 1
int bh_measure_peak(int kind, double* tflops);

/* Stable radix sort that allocates nothing.  The paper has no counterpart:
 * this is the sort of bh_build_tree (Sec. 4.2 step 3a, same kernels, same
 * result) offered on its own to callers that must not allocate device
 * memory here, e.g. code whose device memory is all handed to its own pool
 * allocator (so a cudaMalloc would fail or fragment that pool), or a
 * real-time loop that cannot take the device-wide synchronisation cudaFree
 * implies.  It makes no cudaMalloc/cudaFree call and calls no allocating
 * library routine; its scratch is one fixed array of
 * 4 * (256 * BH_SORT_STATIC_MAX_N / 4096 + 128) bytes (about 1 MiB) in the
 * library's device global memory, one copy per device.
 *
 *  keys      [n] uint64 device, in: keys; out: keys in ascending order.
 *  idx       [n] uint32 device, out: idx[i] = input position of the key now
 *            at i; equal keys keep their input order (stable).
 *  keys_tmp, idx_tmp  [n] caller-owned device scratch, contents clobbered.
 *            The four buffers must be pairwise disjoint byte ranges
 *            (any overlap is rejected with BH_E_INVAL).
 *  n         0 <= n <= BH_SORT_STATIC_MAX_N; larger n is rejected with
 *            BH_E_INVAL before anything runs.
 *  stream    cudaStream_t for all work (NULL = legacy default stream).  The
 *            call only enqueues work and returns; it does not synchronise.
 *  err, err_len  optional caller buffer for a message on failure (NULL ok).
 * All eight 8-bit passes run, so all 64 key bits are sorted.
 * The first call on each device does set-up with that device current: it
 * looks up the scratch array's address (cudaGetSymbolAddress) and sets the
 * sort kernel's shared-memory limit; make that first call before capturing
 * any stream on that device.  The looked-up address belongs to the device's
 * primary context: after cudaDeviceReset (or anything else that destroys
 * that context) this entry point must not be called again in the process.
 * Every call on one device uses the same scratch
 * array, so calls that can overlap in time (different streams or host
 * threads) race and give wrong results: order them, e.g. on one stream.
 * Errors: BH_E_INVAL (n out of range, NULL or overlapping buffers, device
 * ordinal >= 64), BH_E_CUDA (set-up or launch failure). */
#define BH_SORT_STATIC_MAX_N 4194304
int bh_sort_keys_static(uint64_t* keys, uint32_t* idx, uint64_t* keys_tmp, uint32_t* idx_tmp, int64_t n,
                        void* stream, char* err, size_t err_len);

/* The FP64 -> FP32 hi/lo split the FP32 path applies to every particle
 * coordinate and mass each evaluation (Sec. 4.7: the single-precision
 * kernel works on coordinates relative to a group origin, formed from these
 * pairs), on its own: hi[i] = v[i] rounded to the nearest float (ties to
 * even), lo[i] = v[i] - hi[i] (exact in FP64) rounded the same way.  Every
 * finite or non-finite input gives the bits of those two conversions.
 *
 *  v       [n] double, device, in.
 *  hi, lo  [n] float, device, out; caller-owned, distinct, not overlapping v.
 *  n       >= 0.
 *  stream  cudaStream_t (NULL = legacy default stream); enqueues one kernel
 *          and returns without synchronising.
 * No context is needed and nothing is allocated.  Errors: BH_E_INVAL (n < 0,
 * a NULL pointer with n > 0, hi == lo), BH_E_CUDA (launch failure). */
int bh_split_f32(const double* v, float* hi, float* lo, int64_t n, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BH_H */
