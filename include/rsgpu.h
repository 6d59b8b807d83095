/*
 * rsgpu.h -- C ABI of the GB300 ROCKSTAR hot path.
 *
 * The library finds dark-matter halos in a periodic box of particles the way
 * the ROCKSTAR halo finder does (Behroozi, Wechsler & Wu, arXiv:1110.4372):
 *
 *   rs_fof3d       3D friends-of-friends over the box                Sec. 3.1
 *   rs_fof3d_accel the paper's accelerated variant of it             Sec. 3.1
 *   rs_group_sort  groups of at least min_n particles as a CSR list  Sec. 3.1, App. A
 *   rs_refine6d    phase-space FOF hierarchy inside every group      Sec. 3.2, Eq. 1
 *   rs_refine6d_sampled  the same with subset linking lengths        Sec. 3.2
 *   rs_assign      seeds, seed merge and particle assignment         Sec. 3.3, Eqs. 2-4
 *   rs_halo_props  halo centres and the host/subhalo relation        Sec. 3.4, 3.5.1
 *   rs_unbind      single-pass unbinding                             Sec. 3.4, App. B
 *   rs_find_halos  rs_fof3d, rs_group_sort, rs_refine6d(_sampled) and rs_assign
 *                  in sequence, with host or device buffers
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * Pointers.    Array arguments are DEVICE pointers owned by the caller unless
 *              stated otherwise.  Positions and velocities are float32, n rows
 *              of `stride` floats (stride 3 or 4; x, y, z first).  Positions
 *              lie in [0, box); velocities are in any unit.
 * Streams.     All device work is enqueued on the context's stream.  Calls
 *              that return host scalars synchronise that stream first.
 * Errors.      No call aborts, traps or prints.  Every call returns an
 *              rs_status; rs_last_error() gives a one-line message for the
 *              last failure on that context.  Device-side failures (a bounded
 *              wait that ran out, a table that overflowed) are recorded in a
 *              device status word and reported by the next synchronising call.
 * Sizes.       n < 2^31 (RS_ERR_TOO_LARGE otherwise).  n = 0 is valid.
 * Memory.      The context owns a grow-only device workspace allocated with
 *              cudaMalloc and freed by rs_destroy.  rs_tree objects are owned
 *              by the library and freed by rs_tree_free.
 * Threads.     A context may be used by one host thread at a time.
 */
#ifndef RSGPU_H
#define RSGPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RS_OK = 0,
    RS_ERR_INVALID_ARG = 1, /* a size, pointer, stride or parameter is out of range */
    RS_ERR_CUDA = 2,        /* a CUDA runtime call failed (message in rs_last_error) */
    RS_ERR_OOM = 3,         /* device allocation failed */
    RS_ERR_TIMEOUT = 4,     /* a bounded device-side wait ran out; results are invalid */
    RS_ERR_TOO_LARGE = 5,   /* n >= 2^31, or a grid or table would exceed its index range */
    RS_ERR_INTERNAL = 6,    /* an internal capacity or consistency check failed */
    RS_ERR_EXTENT = 7       /* a group spans half the box or more on some axis */
} rs_status;

typedef struct rs_ctx rs_ctx;
typedef struct rs_tree rs_tree;
typedef struct rs_halos rs_halos;

/* Parameters of the method (Table 2 of the paper, plus the merge threshold
 * of Eq. 2 and the virial overdensity of Sec. 3.3). */
typedef struct {
    double b;            /* 3D linking length in units of the mean interparticle spacing (0.28) */
    double f;            /* fraction of a node's particles linked at each level (0.7), 0 < f < 1 */
    int32_t min_n;       /* smallest subgroup kept (10), >= 2 */
    double delta_vir;    /* rho_vir / rho_background for r_dyn,vir (360) */
    double nbar;         /* background number density; <= 0 means n / box^3 */
    double merge_thresh; /* seeds merge below this Eq. 2 separation (10 sqrt 2) */
    int64_t nn_subset;   /* 0: every member's nearest neighbour sets a node's linking length;
                            else nodes above this many members use a random subset of this
                            size (the paper uses 10,000, Sec. 3.2); 0 or in [1024, 2^31) */
    uint64_t nn_seed;    /* seed of that subset (see rs_refine6d_sampled) */
} rs_params;

/* Fills p with the paper's defaults: b = 0.28, f = 0.7, min_n = 10,
 * delta_vir = 360, nbar = 0 (derived), merge_thresh = 10 sqrt 2, and the
 * exact linking length (nn_subset = 0, nn_seed = 0). */
void rs_params_default(rs_params *p);

/* Creates a context bound to a CUDA stream (a cudaStream_t cast to void*;
 * NULL = the legacy default stream) on the current device. */
rs_status rs_create(rs_ctx **out, void *cuda_stream);
void rs_destroy(rs_ctx *ctx);
rs_status rs_set_stream(rs_ctx *ctx, void *cuda_stream);
const char *rs_status_string(rs_status s);
const char *rs_last_error(const rs_ctx *ctx);

/* Launch choices per size class, picked by measurement.  None of them
 * changes a result: every setting computes the same partitions, linking
 * lengths and halo ids (only which CTA or warp does which work, and in
 * which order).  A context starts with rs_tuning_default's values, which
 * are the ones the library's tuner chose on a GB300 (the tuner, its
 * coordinate descent and its result check are in the Python package).
 *   link_blocks_per_sm  big-node link search: resident warps per SM the
 *                       kernel is compiled for, in units of eight (4, 5 or 6:
 *                       32, 40 or 48 warps);
 *   nn_blocks_per_sm    big-node nearest-neighbour search, the same (5, 6
 *                       or 7);
 *   kd_levels           big-node levels whose members are put in k-d order
 *                       (0-3; deeper levels keep their parent's order);
 *   bracket_min         big nodes above this many members search with the
 *                       sampled bracket of the linking length (>= 1024);
 *   mid_max             subtrees of at most this many members run in the
 *                       128-thread tier (33-256); larger ones up to 1024 run
 *                       in the 256-thread tier;
 *   tiny_max            subtrees of at most this many members run one per
 *                       warp (10-32);
 *   small_ctas_per_sm, mid_ctas_per_sm, tiny_ctas_per_sm
 *                       persistent CTAs per SM of the three subtree tiers
 *                       (1-2, 1-8, 1-16);
 *   fof_link_ctas_per_sm  CTAs per SM of the grid-stride 3D link (1-64). */
typedef struct {
    int32_t link_blocks_per_sm;
    int32_t nn_blocks_per_sm;
    int32_t kd_levels;
    int32_t bracket_min;
    int32_t mid_max;
    int32_t tiny_max;
    int32_t small_ctas_per_sm;
    int32_t mid_ctas_per_sm;
    int32_t tiny_ctas_per_sm;
    int32_t fof_link_ctas_per_sm;
} rs_tuning;

void rs_tuning_default(rs_tuning *t);
/* RS_ERR_INVALID_ARG (and no change) if a field is outside its range. */
rs_status rs_set_tuning(rs_ctx *ctx, const rs_tuning *t);
rs_status rs_get_tuning(const rs_ctx *ctx, rs_tuning *t);

/* Failure-detection self-test.  One device thread waits, at most limit polls
 * (1 <= limit <= 2^24, about 0.1 us each), for a flag that only it can set,
 * and sets it first when set_flag is nonzero.  A wait that runs out is
 * recorded in the device status word like every bounded wait of the library,
 * and this synchronising call returns RS_ERR_TIMEOUT; the status word is then
 * clear and the context usable.  With set_flag the call returns RS_OK. */
rs_status rs_selftest_wait(rs_ctx *ctx, int32_t set_flag, int64_t limit);

/* Sec. 3.1: the linking length b times the cube root of the mean volume per
 * particle, l = b * cbrt(box^3 / n), in float64.  0 for n = 0. */
double rs_linking_length(int64_t n, double box, double b);

/* ------------------------------------------------------------------------ */
/* 3D friends-of-friends (Sec. 3.1)                                          */
/* ------------------------------------------------------------------------ */
/* Two particles are friends when their periodic (minimum-image) distance is
 * at most l = rs_linking_length(n, box, b); groups are the connected
 * components.  Writes labels[i] = the smallest particle index in i's group
 * (device, n int32).  Distances are tested in float32 and every pair within
 * a proven float32 error band of l is re-tested in float64, so the partition
 * equals the float64 one.
 *   n_groups  (host, optional) number of groups, singletons included;
 *   n_tieband (host, optional) number of pairs with |d - l| <= 1e-6 l; asking
 *             for it runs an extra pass over every pair within 2 l.
 * Passing either host pointer synchronises.  Errors: RS_ERR_INVALID_ARG for
 * box <= 0, b <= 0, stride not 3 or 4, a box narrower than about seven
 * linking lengths, or a box below 14 linking lengths for which no grid of
 * 4k cells per side has cells between l/2 and l/sqrt 3 (box/l in 4.6-6.4,
 * 6.9-8.1, 9.2-10.1, 11.5-12.1 or 13.9-14.1, roughly); RS_ERR_TOO_LARGE for
 * n >= 2^31 or more than 2^32 grid cells of side 4 l / sqrt 3. */
rs_status rs_fof3d(rs_ctx *ctx, const float *pos, int32_t stride, int64_t n, double box, double b,
                   int32_t *labels, int64_t *n_groups, int64_t *n_tieband);

/* The paper's accelerated 3D FOF (Sec. 3.1): a particle with more than
 * dense_n other particles within l (the paper's 16) is joined with every
 * particle within 2l, and the neighbour search of its neighbours within l is
 * skipped.  Particles are taken in index order, which gives the closed form
 * computed here: a dense particle is a "centre" when no centre of smaller
 * index lies within l; groups are the components of the plain FOF graph
 * plus an edge from every centre to every particle within 2l (inclusive).
 * Every group is a union of plain FOF groups.  labels as rs_fof3d (device,
 * n int32).  n_groups and n_centres (host, optional; n_centres = number of
 * centres) synchronise.  The call always synchronises once per round of the
 * centre choice.  Errors as rs_fof3d; RS_ERR_INVALID_ARG for dense_n < 0;
 * RS_ERR_INTERNAL if the centre choice has not settled after 65536 rounds. */
rs_status rs_fof3d_accel(rs_ctx *ctx, const float *pos, int32_t stride, int64_t n, double box, double b,
                         int32_t dense_n, int32_t *labels, int64_t *n_groups, int64_t *n_centres);

/* Groups with at least min_n members as a CSR list -- the work units of
 * App. A.  perm (device, capacity n) receives the members of each such group
 * back to back, groups ordered by label, members ascending; offsets (device,
 * capacity offsets_cap) receives n_groups + 1 int64 boundaries.  n_groups and
 * n_members (host) are required; the call synchronises.  RS_ERR_INTERNAL if
 * offsets_cap < n_groups + 1 (n_groups is still written). */
rs_status rs_group_sort(rs_ctx *ctx, const int32_t *labels, int64_t n, int32_t min_n, int32_t *perm,
                        int64_t *offsets, int64_t offsets_cap, int64_t *n_groups, int64_t *n_members);

/* rs_fof3d without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * when they need groups -- a plugin inside a host framework whose own pool
 * allocator owns the device memory, a service that fixes its device memory
 * budget at start-up, or a latency-critical loop that must not stall on an
 * allocator or run out of memory mid-run.
 *
 * It writes the same labels as rs_fof3d (device pointers pos and labels,
 * owned by the caller; work enqueued on cuda_stream, NULL = legacy default
 * stream) and synchronises that stream before returning.  Every temporary
 * lives in one fixed scratch array of about 10 MB inside the library image,
 * which every GPU that loads the library holds until the process exits.
 * Limits: at most 65536 particles, and a neighbour table of at most 2^20
 * cells (about 7 linking lengths times 2^(20/3) per box side); beyond either,
 * RS_ERR_TOO_LARGE and nothing runs.  Other errors as rs_fof3d (status code
 * only; there is no context for a message).
 *
 * The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current.  Every call synchronises
 * cuda_stream before it returns (it reads the device status word), so no
 * call can be made while that stream is being captured into a CUDA graph.
 * All calls share the one array and it keeps the last call's contents: calls
 * that overlap on the GPU (from different streams or host threads) race on
 * it and give wrong results. */
rs_status rs_fof3d_static(const float *pos, int32_t stride, int64_t n, double box, double b, int32_t *labels,
                          void *cuda_stream);

/* ------------------------------------------------------------------------ */
/* Phase-space hierarchy (Sec. 3.2, Eq. 1)                                   */
/* ------------------------------------------------------------------------ */
/* For every group g (members perm[group_offsets[g] .. group_offsets[g+1]),
 * device) with at least min_n members: normalise positions and velocities by
 * the node's dispersions sigma_x, sigma_v (3D totals, 1/n), find each
 * member's nearest neighbour under Eq. 1, set the linking length to the k-th
 * smallest nearest-neighbour distance with k = ceil(f n), take the connected
 * components at that length, keep components of at least min_n members
 * (and fewer than the node's) as children, and recurse.  Nodes without
 * children are the seed halos.  Means are accumulated exactly in 64-bit
 * fixed point, distances in float32 with a float64 recheck of every pair in
 * the float32 error band of a linking length, so every partition equals the
 * float64 one.  *out receives a library-owned tree (free with rs_tree_free).
 * Synchronises.  RS_ERR_EXTENT if a node spans half the box on some axis. */
rs_status rs_refine6d(rs_ctx *ctx, const float *pos, const float *vel, int32_t stride, int64_t n, double box,
                      const int32_t *perm, const int64_t *group_offsets, int64_t n_groups, double f,
                      int32_t min_n, rs_tree **out);

/* rs_refine6d with the paper's subsampled linking length (Sec. 3.2: in
 * groups above 10,000 particles the nearest neighbours of a random 10,000-
 * particle subset set the linking length).  A node with more than subset_n
 * members computes the nearest-neighbour distance (among all its members)
 * of subset_n of them only, and its linking length is the k-th smallest of
 * those with k = ceil(f subset_n); linking still uses every pair.  The subset
 * is the subset_n members with the smallest keys, particle i's key being the
 * SplitMix64 output (Steele, Lea & Flood 2014) for the counter
 * subset_seed + (i+1) * 0x9e3779b97f4a7c15: z ^= z >> 30; z *= 0xbf58476d1ce4e5b9;
 * z ^= z >> 27; z *= 0x94d049bb133111eb; z ^= z >> 31 (all mod 2^64).  Keys
 * are distinct, so the subset is unique and the result deterministic.
 * subset_n = 0 is rs_refine6d.  RS_ERR_INVALID_ARG unless subset_n is 0 or in
 * [1024, 2^31).  Everything else as rs_refine6d. */
rs_status rs_refine6d_sampled(rs_ctx *ctx, const float *pos, const float *vel, int32_t stride, int64_t n,
                              double box, const int32_t *perm, const int64_t *group_offsets, int64_t n_groups,
                              double f, int32_t min_n, int64_t subset_n, uint64_t subset_seed, rs_tree **out);

/* Host scalars of a tree: node count, number of levels (max level + 1),
 * seed (leaf) count, tie-band pairs over all nodes, member count (the sum of
 * the refined groups' sizes).  Any pointer may be NULL. */
rs_status rs_tree_info(const rs_tree *t, int64_t *n_nodes, int32_t *n_levels, int64_t *n_seeds,
                       int64_t *n_tieband, int64_t *n_members);

/* Node table, device outputs of n_nodes entries (xbar, vbar: 3 per node),
 * each pointer optional (NULL = skip).  Members of node i are
 * members[first[i] .. first[i] + count[i]) of rs_tree_members, its children's
 * members at the front of that range (nested intervals).  lnk is the linking
 * length in units of the node's own metric (Eq. 1); xbar is wrapped into
 * [0, box); minidx is the smallest member particle index; tie counts the
 * node's tie-band pairs (|d - l| <= 1e-6 l, d != l). */
rs_status rs_tree_nodes(rs_ctx *ctx, const rs_tree *t, int32_t *parent, int32_t *level, int64_t *first,
                        int64_t *count, int32_t *minidx, int32_t *nchild, double *lnk, double *xbar,
                        double *vbar, double *sigx, double *sigv, int64_t *tie);

/* Member particle indices in tree order (device, n_members int32). */
rs_status rs_tree_members(rs_ctx *ctx, const rs_tree *t, int32_t *members);

/* labels[i] (device, n int32) = the smallest member index of the node at
 * `level` that holds particle i, or -1. */
rs_status rs_tree_level_labels(rs_ctx *ctx, const rs_tree *t, int32_t level, int64_t n, int32_t *labels);

void rs_tree_free(rs_tree *t);

/* ------------------------------------------------------------------------ */
/* Seeds, merge and assignment (Sec. 3.3, Eqs. 2-4)                           */
/* ------------------------------------------------------------------------ */
/* Seeds are the tree's leaves.  Within each 3D group two seeds merge when
 * Eq. 2 with the smaller seed's Poisson uncertainties sigma/sqrt(n) is below
 * params->merge_thresh (merges close transitively).  A halo's id is the
 * smallest particle index among its seeds' members; its centre, bulk
 * velocity, sigma_v and v_max come from those members, and r_dyn,vir
 * (Eq. 4) = v_max / sqrt(4/3 pi G rho_vir) with rho_vir = delta_vir m nbar.
 * Each particle is decided at the deepest node holding it: a seed's members
 * go to its halo; a node's other members go to its only halo if its seeds
 * form one, else to the halo nearest under Eq. 3 (ties to the smaller id).
 * halo_id (device, n int32) gets the halo id or -1 outside refined groups;
 * n_halos (host, optional) synchronises.  The same pos/vel as rs_refine6d. */
rs_status rs_assign(rs_ctx *ctx, const rs_tree *t, const float *pos, const float *vel, int32_t stride, int64_t n,
                    double box, const rs_params *params, int32_t *halo_id, int64_t *n_halos);

/* rs_assign that also returns the halos: *halos (optional) receives a
 * library-owned table (free with rs_halos_free) of every halo's id, centre
 * and bulk velocity of its seeds' members, sigma_v, r_dyn,vir^2 and 3D
 * group, and every seed's halo, in the assignment's own halo order.  It is
 * the input of rs_halo_props and rs_unbind.  Otherwise as rs_assign. */
rs_status rs_assign_ex(rs_ctx *ctx, const rs_tree *t, const float *pos, const float *vel, int32_t stride, int64_t n,
                       double box, const rs_params *params, int32_t *halo_id, int64_t *n_halos, rs_halos **halos);
void rs_halos_free(rs_halos *h);
/* Number of halos in the table (0 for NULL). */
int64_t rs_halos_count(const rs_halos *h);
/* Copies the table's per-halo values to device arrays of n_halos entries
 * (xbar, vbar: 3 each); any pointer may be NULL. */
rs_status rs_halos_export(rs_ctx *ctx, const rs_halos *h, int32_t *id, double *xbar, double *vbar, double *sigv,
                          double *rdyn2);

/* ------------------------------------------------------------------------ */
/* Halo properties (Sec. 3.4, 3.5.1) and unbinding (Sec. 3.4, App. B)       */
/* ------------------------------------------------------------------------ */
/* Centres and hosts, per halo in the table's order (device outputs of
 * n_halos entries; xc, vc: 3 each).  A node belongs to a halo when all its
 * seeds do; the halo's centre is the mean position and velocity (xc, vc) of
 * its node with the smallest sigma_x / sqrt(n) (Sec. 3.5.1; ties: smaller
 * smallest member, then smaller level), centre_node that node's index.
 * n_assigned counts the particles with the halo's id in halo_id (device, n,
 * from the rs_assign_ex that made the table).  host is the id of the halo of
 * the same 3D group with more assigned particles that is nearest to the
 * centre under Eq. 3 with that halo's centre, velocity, r_dyn,vir and
 * sigma_v (Sec. 3.4; ties to the smaller id), or -1.  Synchronises.
 * RS_ERR_INVALID_ARG if the table is not this tree's or halo_id holds an
 * id the table lacks. */
rs_status rs_halo_props(rs_ctx *ctx, const rs_tree *t, const rs_halos *h, const int32_t *halo_id, int64_t n,
                        int32_t *centre_node, double *xc, double *vc, int64_t *n_assigned, int32_t *host);

/* Single-pass unbinding (Sec. 3.4).  A halo's set is the particles assigned
 * to it or to any halo below it in the host relation (host: device, n_halos
 * ids or -1, e.g. from rs_halo_props); v_bulk is the set's mean velocity.  A
 * particle is bound to the halo when |v - v_bulk|^2 / 2 + phi < 0, with the
 * potential per unit mass phi = -gm sum_j (r_ij^2 + eps^2)^(-1/2) over the
 * rest of the set (periodic minimum image; gm = G times the particle mass in
 * (velocity unit)^2 x (position unit); with eps = 0 coincident pairs are left
 * out).  theta = 0: phi is summed directly for every set (float32 pair terms,
 * float64 sums of 256-term chunks).  0 < theta < 1: sets above 4096 members
 * use a tree in which a box of particles with mass centre x0, sigma^2 and
 * r_max stands for them beyond d(theta) = r_max/2 + sqrt((r_max/2)^2 +
 * sigma^2/theta) (App. B; the paper's accuracy is 4%), so each such phi is
 * within theta |phi| of the direct sum.  Device outputs: n_part, n_bound
 * (n_halos int64), vbulk (3 per halo), bound_own (n int8: bound to its own
 * halo's set; -1 outside every halo), phi_own (optional, n float64: phi in
 * its own halo's set; untouched outside every halo).  Synchronises.
 * RS_ERR_INVALID_ARG for a cycle in host or theta outside [0, 1). */
rs_status rs_unbind(rs_ctx *ctx, const rs_tree *t, const rs_halos *h, const int32_t *halo_id, const int32_t *host,
                    const float *pos, const float *vel, int32_t stride, int64_t n, double gm, double eps,
                    double theta, int64_t *n_part, int64_t *n_bound, double *vbulk, int8_t *bound_own,
                    double *phi_own);

/* ------------------------------------------------------------------------ */
/* Whole path                                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n_fof_groups;   /* 3D groups with >= min_n members */
    int64_t n_members;      /* particles in those groups */
    int64_t n_nodes;        /* hierarchy nodes */
    int32_t n_levels;
    int64_t n_seeds;
    int64_t n_halos;
    int64_t n_tieband6d;
    int64_t sum_level_members; /* members summed over all nodes (for byte counts) */
    int64_t sum_big_level_members; /* the part of it processed by the multi-block level path */
    int32_t n_fallback_levels;     /* big-node levels whose sampled search radius did not hold */
} rs_stats;

/* rs_fof3d + rs_group_sort + rs_refine6d + rs_assign.  With host_buffers =
 * 0, pos, vel, fof_labels and halo_id are device pointers; with
 * host_buffers = 1 they are host pointers (pinned memory gives full copy
 * speed): the inputs are copied to the context's workspace and both outputs
 * copied back before the call returns.  The copies overlap the kernels: the
 * positions go first, the velocities travel on a second stream of the
 * context while the 3D FOF and the group sort run, and fof_labels comes back
 * on it while the refinement runs; the caller's buffers must stay valid
 * until the call returns.  Positions, velocities and halo ids in mapped
 * pinned memory with 16-byte aligned addresses are moved by a copy kernel
 * that reads or writes the host buffer in place (other host memory goes
 * through cudaMemcpyAsync).  fof_labels and stats may be NULL.
 * Synchronises. */
rs_status rs_find_halos(rs_ctx *ctx, const float *pos, const float *vel, int32_t stride, int64_t n, double box,
                        const rs_params *params, int32_t *fof_labels, int32_t *halo_id, rs_stats *stats,
                        int32_t host_buffers);

/* ------------------------------------------------------------------------ */
/* Instrumentation                                                           */
/* ------------------------------------------------------------------------ */
/* When enabled, every kernel launch on the context is bracketed by CUDA
 * events on the context's stream; rs_profile_read (synchronises) returns per
 * kernel name the launch count and total device milliseconds. */
rs_status rs_profile_enable(rs_ctx *ctx, int32_t on);
void rs_profile_reset(rs_ctx *ctx);
int32_t rs_profile_count(rs_ctx *ctx);
rs_status rs_profile_read(rs_ctx *ctx, int32_t i, const char **name, int64_t *launches, double *total_ms);
/* Number of kernel launches issued on the context since the last reset
 * (counted whether or not profiling is enabled). */
int64_t rs_launch_count(const rs_ctx *ctx);
/* Bytes of device workspace the context holds now.  The workspace grows to
 * the largest call seen; when the device runs out of memory, the scratch of
 * the 3D FOF and of the group sort is released while neither runs, and the
 * allocation is retried (the 1.07B-particle path relies on this). */
int64_t rs_workspace_bytes(const rs_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* RSGPU_H */
