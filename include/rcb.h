/*
 * rcb.h -- C ABI of the GB300 (sm_103a) recursive coordinate bisection (RCB) tree for
 * neighbour search and gravity (Gafton & Rosswog 2011).
 *
 * The tree is built once per particle configuration (rcb_build); neighbour search and gravity
 * are then separate calls that can be made independently (Sec. 3.2.2).  All particle indices
 * that enter or leave the library are the caller's original indices.
 *
 * Conventions shared by every entry point
 *   - Pointers marked "device" address global memory on the current CUDA device; pointers
 *     marked "host" address host memory.  Arrays are dense, C order, little endian.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Every
 *     call is ordered on that stream.  A call returns once its work is queued unless its
 *     description says that it synchronises (to read a size back).
 *   - Return value: RCB_OK (0) or a negative RCB_ERR_* code; rcb_strerror() names it.  A
 *     failed call leaves caller buffers in an unspecified state but the tree usable (except
 *     RCB_ERR_CUDA, after which the CUDA context may be unusable).
 *   - No entry point traps, asserts or waits without bound on the device: loops with an open
 *     bound carry an iteration limit and report RCB_ERR_LIMIT instead.
 */
#ifndef RCB_H
#define RCB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RCB_OK 0
#define RCB_ERR_ARG (-1)      /* NaN/Inf input, N < 1 or N >= 2^31, m <= 0, h <= 0, theta < 0,
                                 n_ll < 1, a mass ratio beyond the 62-bit fixed-point range,
                                 NULL where a pointer is required */
#define RCB_ERR_ALLOC (-2)    /* an allocation (callback or cudaMallocAsync) failed */
#define RCB_ERR_CAPACITY (-3) /* a caller-provided output is smaller than needed */
#define RCB_ERR_CUDA (-4)     /* a CUDA runtime call or kernel launch failed */
#define RCB_ERR_LIMIT (-5)    /* a bounded device loop gave up (see the call's description) */
#define RCB_ERR_STATE (-6)    /* the call needs state the tree does not have */

#define RCB_FLAG_TIMING 1u /* record CUDA events around every stage (see rcb_stage_times) */
#define RCB_FLAG_CENTRE_OF_NUMBER 2u /* Sec. 2.1.3 variant: cut every cell through its centre of
                                        number (unit weights) instead of its centre of mass; the
                                        node moments stay mass-weighted */
#define RCB_FLAG_MAC_ONLY 4u /* Sec. 2.5 variant: near lists from the MAC alone (no reachability
                                override), so gravity sees shorter near lists; neighbour
                                candidates come from a reachability walk of their own, and
                                rcb_gravity_neighbours runs gravity and the neighbour count as
                                two passes */

#define RCB_FLAG_MEDIAN_SPLIT 8u /* Sec. 2.1.3 variant: cut every cell at the median position along
                                    its longest side (the coordinate of rank floor(n/2) of its n
                                    particles; x < split goes left, so particles tied with the
                                    median all go right), giving daughters of floor(n/2) and
                                    ceil(n/2) particles when coordinates are distinct; excludes
                                    RCB_FLAG_CENTRE_OF_NUMBER (RCB_ERR_ARG) */

#define RCB_FP64 0  /* gravity in FP64 throughout */
#define RCB_MIXED 1 /* FP32 near field on cell-relative offsets with compensated sums; FP32
                       multipole tensors; Taylor coefficients accumulated with compensation
                       and stored in FP64 (the build is identical in both forms) */

/* Build parameters. */
typedef struct {
    int32_t n_ll;      /* target mean occupancy of the lowest-level cells, Sec. 2.1.1
                          (paper default 12); the depth L is the smallest L >= 1 with
                          N < n_ll * 2^L (Table 1) */
    int32_t precision; /* RCB_FP64 or RCB_MIXED: form used by rcb_gravity and the backward */
    double theta;      /* opening angle of the geometric MAC, Eq. 4 (theta = 0: direct sum) */
    uint32_t flags;    /* 0 or an OR of the RCB_FLAG_* bits above */
    uint32_t reserved;
} rcb_params;

/* Optional device-memory allocator (for example a caching allocator).  `alloc` returns device
 * memory of at least `bytes` bytes usable on `stream`, or NULL; `release` returns it.  If both
 * are NULL the library uses cudaMallocAsync / cudaFreeAsync on the call's stream. */
typedef void *(*rcb_alloc_fn)(size_t bytes, void *ctx, void *stream);
typedef void (*rcb_free_fn)(void *ptr, void *ctx, void *stream);

/* Opaque tree.  It owns every internal array (sorted particle copies, node moments, interaction
 * lists), allocated through the allocator given to rcb_build and released by rcb_free. */
typedef struct rcb_tree rcb_tree;

/*
 * rcb_build -- Sec. 2.1 tree build and Sec. 2.2-2.4.1 interaction lists.
 *   Splits the root cell level by level through each cell's centre of mass along its longest
 *   side (Sec. 2.1.3; or through its centre of number, or at its median position, as the
 *   RCB_FLAG_* split bits select), partitioning each cell's particles (Sec. 2.1.4), down to level
 *   L; computes per node mass, centre of mass, tight bounding box, geometric centre, size,
 *   traceless quadrupole (Eq. 1, shifted up by Eq. 2), h_node and h_node_int (Sec. 2.3.1);
 *   then walks the tree once per non-empty lowest-level cell (sink) from node 2 and stores its
 *   near list (reachable cells, Sec. 2.3.1, and MAC-rejected ll-cells, Sec. 2.4.1) and far list
 *   (MAC-accepted cells, Eq. 4).
 *   x       device, [N][3] float64 positions (original order)
 *   m, h    device, [N] float64 masses (> 0) and smoothing lengths (> 0)
 *   N       1 <= N < 2^31
 *   params  host, see rcb_params
 *   alloc, release, ctx   optional allocator (both NULL: cudaMallocAsync)
 *   tree    host, in/out: *tree == NULL builds a new tree; a tree from an earlier call is
 *           rebuilt in place, reusing its memory where the sizes allow.
 *   The inputs are copied; the caller may change or free them after the call returns.
 *   The split variants allocate extra memory: N float64 unit weights for the centre-of-number
 *   split; 1 KB of digit histograms per cell larger than 1024 particles (at most N / 1025 + 2
 *   cells) for the median split.
 *   Synchronises `stream` (the list capacities are read back).  Errors: RCB_ERR_ARG (invalid
 *   input, an unknown flag bit or both split bits; *tree unchanged if it was NULL),
 *   RCB_ERR_ALLOC, RCB_ERR_CUDA, RCB_ERR_LIMIT.
 */
int rcb_build(const double *x, const double *m, const double *h, int64_t N, const rcb_params *params,
              rcb_alloc_fn alloc, rcb_free_fn release, void *ctx, void *stream, rcb_tree **tree);

/*
 * rcb_neighbours -- Sec. 2.3: neighbour lists culled from the reachable cells.
 *   Row a holds every b != a with |r_a - r_b| < 2 h_a (FP64 with rounding after every
 *   operation), sorted by original index; rows are in original order (CSR).
 *   offsets  device, [N+1] int64, written: row a is idx[offsets[a] .. offsets[a+1])
 *   idx      device, [capacity] int32 neighbour original indices, or NULL to only count
 *   capacity number of entries idx can hold
 *   needed   host, out: total number of neighbours (offsets[N])
 *   Synchronises `stream`.  Returns RCB_ERR_CAPACITY (offsets and *needed written, idx
 *   untouched) if idx != NULL and capacity < needed.
 */
int rcb_neighbours(rcb_tree *tree, int64_t *offsets, int32_t *idx, int64_t capacity, int64_t *needed,
                   void *stream);

/*
 * rcb_gravity -- Sec. 2.4: near field by kernel-softened direct summation over the near list
 *   (Eqs. 9-10, h = (h_a + h_b)/2, potential phi with phi' = S and phi = -1/r for q >= 2) plus
 *   far field from monopole + quadrupole (Eq. 5) expanded to third order about each sink's
 *   centre of mass (Eq. 6).  G = 1.
 *   acc  device, [N][3] float64 accelerations (original order)
 *   pot  device, [N] float64 potentials, or NULL
 *   Uses the tree's precision (rcb_params.precision or rcb_set_precision).
 */
int rcb_gravity(rcb_tree *tree, double *acc, double *pot, void *stream);

/*
 * rcb_gravity_neighbours -- rcb_gravity and the counting half of rcb_neighbours in one call
 *   (Sec. 2.3 and Sec. 2.4 over the same near list).  In the mixed form one kernel stages each
 *   sink's near-list particles once, evaluates the near field and tests the candidate pairs for
 *   |r_a - r_b| < 2 h_a (the same exact decisions as rcb_neighbours); the FP64 form runs the two
 *   passes one after the other.
 *   acc, pot  as for rcb_gravity
 *   offsets   device, [N + 1] int64, written as rcb_neighbours writes it
 *   needed    host, the total number of neighbour entries
 *   A following rcb_neighbours call with the same tree writes the index list without counting
 *   again (until the next rcb_build or rcb_refit).
 */
int rcb_gravity_neighbours(rcb_tree *tree, double *acc, double *pot, int64_t *offsets, int64_t *needed,
                           void *stream);

/*
 * rcb_gravity_backward -- vector-Jacobian product of rcb_gravity with respect to positions and
 *   masses, with the tree's particle sets and interaction lists held fixed (no paper
 *   counterpart; the forward it differentiates is Sec. 2.4).  Node moments are differentiated
 *   as functions of the particles (Eq. 1, Eq. 2, centre of mass); near-field pair terms are
 *   recomputed, not stored.  Smoothing lengths are constants.
 *   g_acc  device, [N][3] float64 dL/d acc;  g_pot device, [N] float64 dL/d pot, or NULL
 *   g_x    device, [N][3] float64 out;       g_m   device, [N] float64 out
 *   The first call after a build also builds the transposed lists it needs.
 */
int rcb_gravity_backward(rcb_tree *tree, const double *g_acc, const double *g_pot, double *g_x, double *g_m,
                         void *stream);

/*
 * rcb_refit -- Sec. 2.1.8 tree update: new positions and masses (original order, device) for
 *   the same particles.  Node moments, boxes and radii are recomputed bottom-up with the particle
 *   sets and interaction lists unchanged (no re-tessellation, no new walk).  Returns
 *   RCB_ERR_ARG on invalid input.
 */
int rcb_refit(rcb_tree *tree, const double *x, const double *m, void *stream);

/*
 * rcb_update -- Sec. 2.1.8 tree update with its integrity check, for the same particles at new
 *   positions (a time step).  A particle is still in its ll-cell when, at its new position, it
 *   lies on the side of every ancestor's split plane that it was sorted to (x_axis < split for a
 *   left child, not less for a right child; only planes with particles on both sides count;
 *   non-finite coordinates count as outside).
 *   - every particle inside: the smoothing lengths are replaced, the moments, boxes and radii
 *     refitted bottom-up (as rcb_refit) and the tree walked again, so the interaction lists
 *     follow the new positions; the splits stay as built.
 *   - otherwise: the tree is rebuilt in place (as rcb_build on the same handle, with its
 *     parameters and allocator).
 *   x  device, [N][3] float64, original order;  m, h  device, [N] float64
 *   rebuilt  host, may be NULL: 1 if the tree was rebuilt, 0 if it was updated
 *   Synchronises `stream`.  Errors: RCB_ERR_ARG (invalid input), RCB_ERR_STATE (no tree), and
 *   those of rcb_build.
 */
int rcb_update(rcb_tree *tree, const double *x, const double *m, const double *h, int32_t *rebuilt, void *stream);

/*
 * rcb_density -- SPH density by summation over the neighbour lists (Sec. 2.3: smoothed
 *   quantities are kernel-weighted sums over the neighbours), with the cubic spline kernel W
 *   of support 2h the paper uses:
 *     rho_a = m_a W(0, h_a) + sum_{b in nb(a)} m_b W(|r_a - r_b|, h_a)
 *   over the tree's current positions, masses and smoothing lengths (those of the last
 *   rcb_build, rcb_refit or rcb_update).
 *   offsets, idx  device, the CSR written by rcb_neighbours for this tree (original order)
 *   rho           device, [N] float64 out, original order
 *   Pair offsets and W in float32 on a float32 pair split of the positions; the result is
 *   float64.  Does not synchronise.  Errors: RCB_ERR_ARG, RCB_ERR_ALLOC (scratch of 32 B per
 *   particle, allocated on first use through the tree's allocator).
 */
int rcb_density(rcb_tree *tree, const int64_t *offsets, const int32_t *idx, double *rho, void *stream);

/*
 * rcb_neighbour_offsets_noalloc -- the paper has no counterpart: this is a convenience for
 *   callers that cannot allocate device memory when they need neighbour offsets (for example an
 *   application whose memory manager owns the whole device and forbids allocations by libraries).
 *   It returns the same offsets as rcb_neighbours(tree, offsets, NULL, 0, needed, stream) and
 *   allocates nothing: the per-particle counts are written straight into `offsets` and the only
 *   other scratch (the scan's per-tile sums and the status words) is a fixed static array of
 *   about 33 KB inside the library, which every GPU that loads the library keeps until the
 *   process exits.
 *   offsets  device, [N+1] int64, written;  needed  host, out: offsets[N]
 *   Limit: N <= 33,554,432 (2^25); larger trees return RCB_ERR_CAPACITY.
 *   The first call on a device looks the static array up (cudaGetSymbolAddress) with that
 *   device current and keeps its address for the life of the process (the device's primary
 *   context must stay alive: no cudaDeviceReset in between).  All calls share the one array, so
 *   calls that overlap on the GPU (other streams, other threads) race: serialise them.
 *   The call reads the total back to the host and synchronises `stream` before it returns.
 */
int rcb_neighbour_offsets_noalloc(rcb_tree *tree, int64_t *offsets, int64_t *needed, void *stream);

/* Select the gravity form (RCB_FP64 or RCB_MIXED) of an existing tree. */
int rcb_set_precision(rcb_tree *tree, int32_t precision);

/*
 * rcb_tree_info -- host, out [16] int64:
 *   0 N, 1 L, 2 number of node slots (2^(L+1), slot 0 unused), 3 number of ll-cells (2^L),
 *   4 number of sinks (non-empty ll-cells), 5 near-list capacity per sink, 6 far-list capacity
 *   per sink, 7 total near entries, 8 total far entries, 9 total reachable near entries,
 *   10 walk decisions settled in FP64 (after the FP32 filter was inconclusive),
 *   11 number of subtrees built in shared memory, 12 precision, 13 near-field pair count
 *   (sum over sinks of sink particles x near-list particles, self pairs included),
 *   14 neighbour-candidate pair count (the same over reachable cells), 15 number of kernel
 *   launches issued by the library in this process so far.
 */
int rcb_tree_info(const rcb_tree *tree, int64_t *info);

/*
 * rcb_export_topology -- host copies for parity tests (any pointer may be NULL).  Node arrays
 *   are indexed by heap label (Sec. 2.1.5), [2^(L+1)] entries, slot 0 unused.
 *   leaf_of   [N] int32: ll-cell number (0 .. 2^L - 1) of each particle, original order
 *   perm      [N] int32: original index of the particle at each sorted position
 *   first, count [nn] int64; axis [nn] int32; split [nn] float64 (internal nodes)
 *   sums      [nn][4][2] int64: exact sums (mass, m x, m y, m z) as (low, high) 64-bit words
 *   mass [nn]; com [nn][3]; bmin, bmax [nn][3]; rg [nn][3]; H [nn]; hint [nn]; hnode [nn];
 *   Q [nn][6] (xx, xy, xz, yy, yz, zz) -- all float64
 *   Synchronises `stream`.
 */
int rcb_export_topology(rcb_tree *tree, int32_t *leaf_of, int32_t *perm, int64_t *first, int64_t *count,
                        int32_t *axis, double *split, int64_t *sums, double *mass, double *com, double *bmin,
                        double *bmax, double *rg, double *H, double *hint, double *hnode, double *Q,
                        void *stream);

/*
 * rcb_export_lists -- host copies of the interaction lists as CSR over ll-cells j = 0 .. 2^L-1
 *   (node 2^L + j; empty cells have empty lists).  Within a sink's near list the reachable
 *   cells come first; order is otherwise unspecified (compare as sets).
 *   near_off [2^L + 1] int64; near_ids [cap_near] int32 node labels; near_reach [cap_near]
 *   uint8 (1 = reachable, i.e. a neighbour candidate); far_off [2^L + 1]; far_ids [cap_far].
 *   Returns RCB_ERR_CAPACITY if a capacity is below the totals of rcb_tree_info.
 */
int rcb_export_lists(rcb_tree *tree, int64_t *near_off, int32_t *near_ids, uint8_t *near_reach, int64_t cap_near,
                     int64_t *far_off, int32_t *far_ids, int64_t cap_far, void *stream);

/*
 * rcb_stage_times -- host, out [16] float64: device time in milliseconds of the last call of
 *   each stage, measured with CUDA events on the call's stream when the tree was built with
 *   RCB_FLAG_TIMING (zeros otherwise):
 *   0 ingest + root, 1 level passes, 2 shared-memory subtrees, 3 leaf moments + bottom-up +
 *   packing, 4 walk, 5 whole build (0..4), 6 neighbour count + scan, 7 neighbour fill,
 *   8 neighbour row sort, 9 far field, 10 near field (+ Taylor evaluation and scatter),
 *   11 backward, 12..15 reserved.  Synchronises `stream`.
 */
int rcb_stage_times(rcb_tree *tree, double *ms, void *stream);

/* Release the tree and everything it owns (NULL is allowed). */
void rcb_free(rcb_tree *tree);

/* Static description of a status code. */
const char *rcb_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* RCB_H */
