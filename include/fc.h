/*
 * fc.h -- C ABI of the GB300 patch-AMR wave-propagation library.
 *
 * The library advances a scalar tracer, q_t + (u q)_x + (v q)_y = 0, on a
 * forest of quadtrees whose leaves carry fixed-size mx x mx patches with mbc
 * ghost layers (Calhoun & Burstedde, arXiv 1703.03116, Sec. 2: "A quadtree
 * layout").  One device store holds every patch of every forest; all
 * numerical work runs in CUDA kernels on the device.
 *
 * Conventions common to every call:
 *  - Every call returns an fc_status; no exception or abort crosses the ABI.
 *    On failure fc_last_error() returns a thread-local message.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls enqueue work on it and return without synchronising,
 *    unless stated otherwise.  An asynchronous device error is reported as
 *    FC_ERR_CUDA by the next call that synchronises.
 *  - Pointers marked "host" are read or written before the call returns.
 *    Pointers marked "device" must stay valid until the stream reaches the
 *    call's work.  The caller keeps ownership of every buffer it passes; the
 *    library owns the forest and all device storage it allocates.
 *  - Field layout for get/set: interior cells only, [leaf][j][i] (i fastest),
 *    leaves in the order of fc_forest_leaves (forest, block, Morton order).
 *    Element type is the forest's dtype (float for FC_F32, double for FC_F64).
 *  - A forest handle is not thread-safe; use one host thread per handle.
 */
#ifndef FC_H
#define FC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fc_forest fc_forest;

typedef enum {
  FC_OK = 0,
  FC_ERR_INVALID_ARG = 1,   /* bad pointer, size, level or enum value            */
  FC_ERR_PRECONDITION = 2,  /* layout not 2:1 balanced, not covering, mbc > mx/4 */
  FC_ERR_OOM = 3,           /* device or host allocation failed                  */
  FC_ERR_CUDA = 4,          /* a CUDA call or kernel failed                      */
  FC_ERR_TIMEOUT = 5,       /* a bounded device wait gave up                     */
  FC_ERR_STATE = 6          /* call not valid in the forest's current state      */
} fc_status;

typedef enum { FC_F32 = 0, FC_F64 = 1 } fc_dtype;
typedef enum {
  FC_DOMAIN_WALLS = 0,
  FC_DOMAIN_PERIODIC = 1,
  FC_DOMAIN_SPHERE = 2,
  FC_DOMAIN_BRICK = 3
} fc_domain;
typedef enum { FC_VEL_CONST = 0, FC_VEL_SWIRL = 1, FC_VEL_ROTATION = 2, FC_VEL_DEFORM = 3 } fc_velocity;

/* Problem description (Sec. 2; Sec. 5.1 "Problem setup").
 *   domain      unit square with walls, periodic unit square, cubed sphere, or
 *               a periodic brick (Sec. 5.1: a brick_nx x brick_ny arrangement
 *               of unit blocks, each an adaptive quadtree; block
 *               b = by * brick_nx + bx sits at [bx, bx+1] x [by, by+1], its
 *               faces meet its neighbours' with the identity orientation,
 *               and the brick's outer faces are periodic).
 *   nforests    independent forests in one store (a batched ensemble); each
 *               forest of a square domain is one block, each forest of the
 *               cubed sphere six blocks (Sec. 2.4): block b is the face of
 *               the cube [-1,1]^3 with outward normal n and block point
 *               (x, y) in [0,1]^2 at n + (2x-1) ex + (2y-1) ey, with
 *               (n; ex, ey) = 0: (+Z; +X, +Y), 1: (-Z; +X, -Y),
 *               2: (+X; +Y, +Z), 3: (-X; -Y, +Z), 4: (+Y; -X, +Z),
 *               5: (-Y; +X, +Z); the grid is equiangular gnomonic (cube
 *               point n + tan((x-1/2) pi/2) ex + tan((y-1/2) pi/2) ey,
 *               projected onto the unit sphere).
 *   mx, mbc     interior cells per side (power of two, 8..64) and ghost layers
 *               (Proposition 1 requires mbc <= mx/4; only mbc = 2 is built).
 *   lmin, lmax  level range; a level-l leaf has edge 2^-l of its block.
 *   dtype       FC_F32 or FC_F64 for the stored field and the update.
 *   vel_kind    FC_VEL_CONST: (u, v) = (vel[0], vel[1]);
 *               FC_VEL_SWIRL: streamfunction sin^2(pi x) sin^2(pi y)
 *               cos(pi t / T) / pi with T = vel[0];
 *               FC_VEL_DEFORM (sphere only, Sec. 5.3's run): the time-
 *               dependent streamfunction psi = k sin^2(rho - 2 pi t/T)
 *               cos^2(theta) cos(pi t/T) - 2 pi sin(theta)/T_f (longitude
 *               rho, latitude theta; k, T, T_f = vel[0], vel[1], vel[2], T
 *               and T_f nonzero), velocity e_r x grad psi; before each
 *               level substep (and global step) the edge volume fluxes of
 *               the level's patches are recomputed for its half time as
 *               psi differences between the edges' end points, formed as
 *               k c (s_b - s_a)(s_b + s_a) - (2 pi/T_f)(Z_b - Z_a) with
 *               s = Y cos(2 pi t/T) - X sin(2 pi t/T), c = cos(pi t/T),
 *               from the grid corners kept per patch (3 (mx+5)^2 doubles);
 *               times the velocity scale.
 *               FC_VEL_ROTATION (sphere only): solid-body rotation
 *               u = omega x X, omega = (vel[0], vel[1], vel[2]).  The sphere
 *               runs the capacity form: FP64 metrics per patch (cell
 *               areas kappa, edge volume fluxes omega . (X_b - X_a) between
 *               the edge's end points), ghost-cell metrics from the patch's
 *               own mapping, area-weighted fine-to-coarse averages, and
 *               corner ghosts beyond a cube vertex set to the mean of the
 *               two edge ghosts next to them.
 *   order       1 (first order) or 2 (second-order wave corrections).
 *   limiter     0 unlimited, 1 MC.
 *   transverse  0 none, 1 fluctuations, 2 fluctuations and corrections.
 *   reflux      0 (the paper's scheme) or 1: conservative correction at
 *               coarse/fine faces and, on the cubed sphere, at cube edges
 *               (see fc_step_multirate). */
typedef struct {
  int domain;
  int nforests;
  int mx, mbc;
  int lmin, lmax;
  int dtype;
  int vel_kind;
  double vel[4];
  int order;
  int limiter;
  int transverse;
  int indicator;  /* regrid indicator: 0 max |grad q| / 2, 1 max q - min q (Sec. 5.1) */
  int smooth;     /* 1: smooth grading of the target levels (Sec. 3.3) */
  int reflux;     /* 1: refluxing at coarse/fine faces (an extension) */
  int brick_nx, brick_ny;  /* FC_DOMAIN_BRICK: blocks per row and column (<= 256 in all) */
} fc_forest_desc;

/* Create a forest from an explicit leaf list (Sec. 2: quadrants identified
 * by tree coordinates and level; only leaves are stored).
 *   leaves   host, nleaves rows of 5 ints (forest, block, level, ix, iy),
 *            0 <= ix, iy < 2^level; any order.
 * The leaves of each forest must tile its blocks exactly and be 2:1 balanced
 * across faces and corners (FC_ERR_PRECONDITION otherwise).  The field is
 * allocated but undefined until fc_forest_set_q.  Synchronous. */
fc_status fc_forest_create(const fc_forest_desc* desc, int nleaves, const int* leaves,
                           fc_forest** out);
fc_status fc_forest_destroy(fc_forest* forest);

/* Pluggable device allocator.  By default every device allocation of the
 * library comes from the device's stream-ordered pool (cudaMallocAsync /
 * cudaFreeAsync on the API call's stream, or the legacy default stream
 * inside fc_forest_create).  fc_set_allocator routes them all through the
 * caller's functions instead (e.g. a framework's caching allocator):
 *   alloc(bytes, stream, user)        returns a device pointer, 256-byte
 *                                     aligned, usable in stream order on
 *                                     `stream` (a cudaStream_t as void*), or
 *                                     NULL (the call then fails FC_ERR_OOM);
 *   release(ptr, bytes, stream, user) takes back a block, in stream order on
 *                                     `stream`; bytes is the size asked for.
 * Both or neither (NULL, NULL restores the pool).  Process-wide; it may be
 * changed only while no forest exists (FC_ERR_STATE otherwise), so every
 * block is released through the functions that allocated it.  The library
 * calls the functions from the thread that calls it, never during a stream
 * capture of its own. */
typedef void* (*fc_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*fc_free_fn)(void* ptr, size_t bytes, void* stream, void* user);
fc_status fc_set_allocator(fc_alloc_fn alloc, fc_free_fn release, void* user);

/* What a forest holds (Sec. 2: the leaves and their levels).
 *   nleaves              leaves of the field layout (a partition: its own)
 *   leaves_per_level[l]  of them, those of level l (0 <= l < FC_INFO_LEVELS)
 *   device_bytes         device memory the forest holds now (store, tables,
 *                        metrics, adjoint buffers once created)
 *   graphs               captured coarse steps (forward and adjoint) held
 *   tuned_buckets        launch-size buckets the autotuner has timed
 *   coarse_entries       face/corner regions of the layout filled from a
 *                        coarser neighbour
 *   coarse_unlisted      of them, those whose coarse neighbour's ghosts the
 *                        update must look up in that neighbour's own table
 *                        entries (the ghosts it reads are not all listed in
 *                        the region's entry: a slower read chain, same
 *                        values).  Reading these two synchronises the
 *                        device (the table is read back). */
#define FC_INFO_LEVELS 21
typedef struct {
  int nleaves, nforests, mx, mbc, lmin, lmax, dtype, domain;
  int leaves_per_level[FC_INFO_LEVELS];
  int64_t device_bytes;
  int graphs, tuned_buckets;
  int coarse_entries, coarse_unlisted;
} fc_info;
fc_status fc_forest_info(const fc_forest* forest, fc_info* out);

/* Number of leaves, and the leaf list (host, n x 5 ints) in field order. */
fc_status fc_forest_num_leaves(const fc_forest* forest, int* n);
fc_status fc_forest_leaves(const fc_forest* forest, int* out);

/* Copy the interior field in or out (layout in the header comment).
 *   on_device  nonzero: `q` is a device pointer (async on `stream`);
 *              zero: `q` is a host pointer (the call synchronises `stream`). */
fc_status fc_forest_set_q(fc_forest* forest, const void* q, int on_device, void* stream);
fc_status fc_forest_get_q(const fc_forest* forest, void* q, int on_device, void* stream);
/* Whole patch arrays with ghosts, (mx+2mbc)^2 per leaf, [leaf][j][i]. */
fc_status fc_forest_get_q_full(const fc_forest* forest, void* q, int on_device, void* stream);

/* Test aid, an executable Prop. 1 (Sec. 2.3: every cell the update's stencil
 * reads is set by a rule of Alg. 1 first): writes `value` (NaN, say) into
 * every ghost cell of the forest's two state buffers and into every cell of
 * its time-interpolation tiles, enqueued on `stream`.  Interiors are left
 * alone, so the next steps must give the same results as without the call;
 * an update that read such a cell before a rule wrote it would carry the
 * value into its result. */
fc_status fc_forest_poison(fc_forest* forest, double value, void* stream);

/* Alg. 1 (update_ghost, Sec. 2.3) on every level: copy from same-size
 * neighbours (Eq. transform), average from fine neighbours (Eq.
 * ghost_coarse), physical boundary conditions, interpolation from coarse
 * neighbours (Eq. ghost_fine), physical boundary conditions again.
 * All levels must hold data at the same time. */
fc_status fc_fill_ghosts(fc_forest* forest, void* stream);

/* One multirate substep of one level (Sec. 4, local time stepping): fill the
 * ghosts of `level` at time t -- data of level-1 are linearly interpolated in
 * time between its states before and after its own last step -- then advance
 * every level-`level` patch from t to t+dt with the wave-propagation update.
 * Levels are driven coarse-first: level+1 takes two substeps of dt/2 after
 * each substep of `level`.  `level` must hold patches' time t. */
fc_status fc_advance_level(fc_forest* forest, int level, double t, double dt, void* stream);

/* One global time step (every level advanced by dt after one Alg. 1 fill). */
fc_status fc_step_global(fc_forest* forest, double t, double dt, void* stream);

/* One coarse multirate step: the coarse-first recursion of fc_advance_level
 * over all levels, 2^(lmax-lmin) substeps of the finest level.
 * With desc.reflux = 1 (not in the paper: Berger and Colella's refluxing),
 * every level substep also records the final fluxes through its patches'
 * faces, and after the two finer substeps that follow a level-l substep of
 * length dt, each level-l cell next to a finer face exchanges the flux its
 * update used, Fc, for the fine fluxes' mean Fbar = 1/4 (sum over the face's
 * two fine cells and the two fine substeps): q += (dt/h)(Fc - Fbar) on a +x
 * or +y face, q += (dt/h)(Fbar - Fc) on a -x or -y face, faces in the order
 * -x, +x, -y, +y.  Total mass is then conserved to rounding.  (In
 * fc_step_global the weight is 1/2: one fine step of the same dt.)  On the
 * cubed sphere the fluxes are volume fluxes (the fine side's weight is the
 * time ratio alone, 1/2 per substep, 1 in fc_step_global), the correction of
 * a cell is dt / kappa of the cell, and every level substep also exchanges
 * the fluxes of the cube edges: each side computes an edge's flux from its
 * own ghost cells, the side on the block of lower index keeps its own, and
 * a cell on the other side takes it in place of its own (the pairing of
 * fc_layout_reflux).  Every update runs the staged or band variant then;
 * fc_advance_level records the fluxes but corrects nothing. */
fc_status fc_step_multirate(fc_forest* forest, double t, double dt_coarse, void* stream);

/* Tag and regrid (Sec. 3.1).  Fills ghosts, computes on the device the
 * per-leaf indicator max 1/2 |(q(i+1,j)-q(i-1,j), q(i,j+1)-q(i,j-1))| (in
 * the field's precision; the square root in FP64), or with desc.indicator =
 * 1 the spread max q - min q of the leaf's interior,
 * refines leaves above tau_refine (below their forest's maximum level
 * lmax_per_forest[f], or desc.lmax when NULL), 2:1 balances by refinement,
 * coarsens families of four leaves all below tau_coarsen whose parent stays
 * balanced (desc.smooth = 1: each leaf's target level -- one finer if above
 * tau_refine, one coarser if below tau_coarsen, else its own -- is first
 * raised to the largest target among the leaves it touches; leaves refine
 * when their graded target is finer, families coarsen when all four graded
 * targets are coarser), and remaps the field on the device (copy; Eq. ghost_fine
 * interpolation for new children; Eq. ghost_coarse averaging for new
 * parents).  *changed (host) receives the number of leaves created plus
 * removed.  Synchronous. */
fc_status fc_tag_regrid(fc_forest* forest, double tau_refine, double tau_coarsen,
                        const int* lmax_per_forest, int* changed, void* stream);

/* The per-leaf indicator alone, into a host array of nleaves doubles. */
fc_status fc_tag(fc_forest* forest, double* delta_host, void* stream);

/* Velocity scale sigma: every edge speed is multiplied by sigma (default 1).
 * It is the scalar parameter of the adjoint's velocity derivative.  A new
 * value drops the captured steps and tapes (their kernels carry the scale)
 * and synchronizes the device; setting the current value changes nothing. */
fc_status fc_set_velocity_scale(fc_forest* forest, double scale);

/* Adjoint of one global time step (the transposes of Alg. 1 and of the
 * wave-propagation update; an extension for differentiation, with no
 * counterpart in the paper; square domains only).  The forest must hold q^n, the state at the start of the
 * step (it is not advanced).  With the step's map q^{n+1} = S(Fill(q^n)),
 *   lam     device, in/out, field layout: on entry dL/dq^{n+1}, on return
 *           dL/dq^n = (dq^{n+1}/dq^n)^T lam, using the piece of the MC
 *           limiter and of the minmod interpolation slopes that q^n selects
 *           (the a.e. derivative);
 *   dscale  device, one double, accumulated: += lam^T dq^{n+1}/dsigma.
 * Kernels: per-level update transposes (shared-memory tiles), then atomic
 * scatters for the interpolation and copy/average transposes, so the
 * rounding order of those sums is not fixed.  Asynchronous on `stream`. */
fc_status fc_adjoint_step_global(fc_forest* forest, double t, double dt, void* lam,
                                 double* dscale, void* stream);

/* Adjoint of one multirate level substep, fc_advance_level(level, t, dt)
 * (Sec. 4 local time stepping; the adjoint is an extension for
 * differentiation with no counterpart in the paper; square domains only).
 * The forest must hold the state the forward call started from -- the
 * current states of every level, the older state of level-1 that its time
 * interpolation reads, and the bookkeeping of the levels' last steps -- as
 * it stands right before that call; it is not advanced (the substep's ghost
 * fill is redone in place, which changes no interior value).  With the
 * substep's map (level's new state) = U(Fill(q_level, q_level+1,
 * (1 - alpha) q_old(level-1) + alpha q(level-1))):
 *   lam      device, in/out, field layout: on entry the adjoint of every
 *            leaf's current state after the call (level's leaves: of its
 *            new state), on return the adjoint of every leaf's current state
 *            before it; the transposes of the level's update, of its ghost
 *            fill (copies, averages, interpolation slopes on the pieces the
 *            forward state selects) and the newer state's alpha share of the
 *            time interpolation are added where they belong;
 *   lam_old  device, nullable, field layout, accumulated: the adjoint of
 *            each leaf's older state (the state before its level's latest
 *            step); this call adds the (1 - alpha) share of level-1's time
 *            interpolation there.  Needed when level > lmin and level-1
 *            has stepped since the field was set (FC_ERR_INVALID_ARG if then
 *            NULL).  Chaining these calls in reverse over a coarse step, a
 *            caller adds lam_old's entries of a level into lam (and clears
 *            them) right after reversing that level's substep: the older
 *            state is the state before it;
 *   dscale   device, one double, accumulated: += lam^T d(new state)/dsigma.
 * Contributions are atomic adds, so their rounding order is not fixed.
 * Asynchronous on `stream`. */
fc_status fc_adjoint_advance(fc_forest* forest, int level, double t, double dt, void* lam,
                             void* lam_old, double* dscale, void* stream);

/* Adjoint of one coarse multirate step (the coarse-first recursion of
 * fc_step_multirate, Sec. 4): the transpose of every level substep -- the
 * update, the level-restricted Alg. 1 fill, the time interpolation
 * q_T = (1 - alpha) q_old + alpha q of the coarser level and the copy q_old = q
 * -- in reverse order, on the pieces the forward state selects.  The forest
 * must hold the state at the step's start time t; the call replays the
 * forward step once on the device (keeping, before each substep, the states
 * of the levels it touches) and leaves the forest at the start state.
 *   lam     device, in/out, field layout: dL/dq(t + dt_coarse) on entry,
 *           dL/dq(t) on return;
 *   dscale  device, one double, accumulated: += lam^T dq/dsigma.
 * Every contribution to an adjoint is an atomic add (the levels' reversed
 * substeps run side by side where their forward substeps could), so the
 * rounding order of those sums is not fixed.
 * Device memory: three adjoint stores plus the kept states (about two
 * stores per substep for the levels it touches), held until the forest is
 * destroyed.  Square domains only (FC_ERR_INVALID_ARG on the sphere).
 * Work runs on `stream`; the call ends by reading the device error word
 * (synchronous). */
fc_status fc_adjoint_step_multirate(fc_forest* forest, double t, double dt_coarse, void* lam,
                                    double* dscale, void* stream);

/* The same adjoint in two halves, for a caller that steps forward again
 * anyway (a checkpointed gradient recomputing a segment of steps):
 * fc_step_multirate_record is fc_step_multirate (the same kernels, the same
 * result bits) that also keeps in tape `slot` what the reverse of the step
 * reads -- each level substep's ghost-filled input tiles and the
 * time-interpolated coarse cells its interpolation used -- and
 * fc_adjoint_step_multirate_taped is the reverse alone, from that tape,
 * with lam and dscale as in fc_adjoint_step_multirate; it neither reads nor
 * changes the forest's state, so a segment recorded forward is reversed in
 * any order of slots.  t and dt_coarse of the reverse are those the step
 * was recorded with (FC_ERR_STATE when the slot holds no step of that
 * length, or was recorded before the layout or the captured steps last
 * changed: a regrid, fc_set_advance_variant, fc_set_limits, ...).
 *   slot  0 <= slot < FC_MAX_TAPE_SLOTS (FC_ERR_INVALID_ARG otherwise).
 * Device memory per slot: the kept tiles of fc_adjoint_step_multirate
 * (without its copy of the start state), held until fc_tape_release or the
 * forest's destruction.  Square domains only, no refluxing (as
 * fc_adjoint_step_multirate).  Work runs on `stream`: the record is
 * asynchronous, as fc_step_multirate (a device error shows at the next call
 * that reads the error word); the reverse ends by reading the device error
 * word (synchronous). */
#define FC_MAX_TAPE_SLOTS 64
fc_status fc_step_multirate_record(fc_forest* forest, double t, double dt_coarse, int slot,
                                   void* stream);
fc_status fc_adjoint_step_multirate_taped(fc_forest* forest, double t, double dt_coarse, int slot,
                                          void* lam, double* dscale, void* stream);
fc_status fc_tape_release(fc_forest* forest);

/* Total mass per forest, sum over leaves of h^2 sum(q) (on the sphere
 * sum(kappa q)), accumulated in FP64
 * on the device in a fixed order.  out: host, nforests doubles.  Synchronous. */
fc_status fc_forest_mass(const fc_forest* forest, double* out, void* stream);

/* Host-only layout services (no device work; usable without a GPU).
 *
 * fc_layout_check: validate a leaf list against `desc` (tiling, levels, 2:1
 * balance across faces and corners).  Returns FC_OK or FC_ERR_PRECONDITION.
 *
 * fc_layout_neighbours: the face/corner neighbour table of Sec. 2.2-2.4 for
 * a valid leaf list.  out: host, nleaves * 8 rows of 6 ints
 *   (kind, n0, n1, a, fx, fy)
 * in the leaves' field order, regions (-x, +x, -y, +y, (-,-), (+,-), (-,+),
 * (+,+)); kind 0 exterior, 1 same size, 2 finer, 3 coarser, 4 corner
 * region beyond a vertex of the cubed sphere (no neighbour); n0/n1 are field
 * indices of the neighbour leaves; (a, fx, fy) encode Eq. (transform)
 * I' = A I + F on level-l global cell indices (a: bit 0 swaps axes, bits 1
 * and 2 negate the first and second output).
 *
 * fc_layout_regrid: the layout that fc_tag_regrid builds from per-leaf
 * indicators `delta` (host, nleaves doubles, field order).  out_leaves:
 * host, capacity `cap` rows of 5 ints; *nout receives the new count
 * (FC_ERR_INVALID_ARG when cap is too small). */
fc_status fc_layout_check(const fc_forest_desc* desc, int nleaves, const int* leaves);
fc_status fc_layout_neighbours(const fc_forest_desc* desc, int nleaves, const int* leaves,
                               int* out);
fc_status fc_layout_regrid(const fc_forest_desc* desc, int nleaves, const int* leaves,
                           const double* delta, double tau_refine, double tau_coarsen,
                           const int* lmax_per_forest, int cap, int* out_leaves, int* nout);
/* fc_layout_reflux: what refluxing exchanges (Berger and Colella's
 * correction, an extension of the paper's scheme), from the neighbour table
 * and its index transforms.  out: host, nleaves * 4 * mx rows of 5 ints
 * (kind, leaf across, its face on the shared edge, j0, j1) per leaf (field
 * order), face (-x, +x, -y, +y) and face cell along the face's axis: kind 1
 * the leaf across is finer (j0, j1: its cells beside the lower and upper half
 * of the cell), 2 the leaf across has the same level and lies across a cube
 * edge on a block of lower index (its flux is the one kept; j0: its cell),
 * 0 nothing (-1 elsewhere); faces 0 -x, 1 +x, 2 -y, 3 +y. */
fc_status fc_layout_reflux(const fc_forest_desc* desc, int nleaves, const int* leaves, int* out);

/* Partitioned layouts (Sec. 3: partitioning, parallel ghost filling).
 *
 * The leaves, in their field (Morton) order, are split into contiguous ranges
 * of equal work, a level-l leaf weighing 2^(l - lmin) (its updates per
 * coarse step); each rank (one process per GPU, or several partitions on
 * one GPU) holds its own leaves plus its mirrors: the leaves of other ranks
 * whose interiors its ghost fills read -- face and corner neighbours of its
 * leaves and, where a neighbour is coarser, that neighbour's same-size and
 * finer neighbours (its copied and averaged ghosts feed the interpolation;
 * Proposition 1 keeps the interpolated ones out of reach).  Every layout
 * array below is in the caller's leaf order.
 *
 * fc_layout_partition (host only): part_out[i] = the rank of leaf i.
 * fc_layout_halo (host only): the mirrors of `rank` under `part`, as
 *   indices into `leaves`, in field order; mirror_out holds up to nleaves.
 * fc_forest_create_part: rank's part of the layout, on the device.  Its
 *   field layout (set_q, get_q, mass, tag, capacity, leaves) covers the
 *   owned leaves only, in field order; the mirrors are held internally.
 *   fc_fill_ghosts, fc_advance_level and fc_step_global update the owned
 *   leaves; after each of them the caller refreshes the mirrors of the
 *   levels that changed (all levels after fc_step_global and after
 *   fc_forest_set_q, level l after fc_advance_level(l, ...)): for every
 *   other rank r, fc_halo_pack(r, level) on the owner and
 *   fc_halo_unpack(owner, level) on r, moving the packed buffer between
 *   them (a device copy, a send/receive, ...), before the next step reads
 *   them.  Stepping every partition this way gives each owned leaf the same
 *   bits as the unpartitioned forest.  fc_step_multirate, fc_tag_regrid and
 *   the adjoint return FC_ERR_STATE on a partition (its layout is fixed);
 *   refluxing is not built for it.
 * fc_halo_count: patches in the exchange with `peer` for `level` (-1: all
 *   levels, level-major), sent from this rank and received by it.
 * fc_halo_pack: device `dst` <- the interiors (mx x mx of the forest's
 *   dtype each, [patch][j][i]) of this rank's patches that `peer` mirrors,
 *   from their current states, ordered by field order; async on `stream`.
 * fc_halo_unpack: the interiors of this rank's mirrors owned by `peer`, in
 *   the same order, <- device `src` (the peer's packed buffer for this
 *   rank); async on `stream`. */
fc_status fc_layout_partition(const fc_forest_desc* desc, int nleaves, const int* leaves,
                              int nranks, int* part_out);
fc_status fc_layout_halo(const fc_forest_desc* desc, int nleaves, const int* leaves,
                         const int* part, int rank, int* nmirror, int* mirror_out);
fc_status fc_forest_create_part(const fc_forest_desc* desc, int nleaves, const int* leaves,
                                const int* part, int rank, fc_forest** out);
fc_status fc_halo_count(const fc_forest* forest, int peer, int level, int* nsend, int* nrecv);
fc_status fc_halo_pack(const fc_forest* forest, int peer, int level, void* dst, void* stream);
fc_status fc_halo_unpack(fc_forest* forest, int peer, int level, const void* src, void* stream);

/* Per-phase device timers (the paper's run-time breakdown, Sec. 5: advance,
 * ghost fill, regrid).  While enabled, every kernel launch of a phase is
 * bracketed by CUDA events on its stream.
 *   phase: 0 advance, 1 ghost fill, 2 regrid/tag/remap, 3 other.
 * fc_timers_read synchronises the forest's pending timed work and returns,
 * for one phase, the summed kernel time in ms, the number of timed launches
 * and the algorithmic bytes those launches must move (advance: every patch
 * array read once with ghosts, every interior written once; fill: every
 * filled ghost cell written once and its source read once).  reset != 0
 * clears the phase afterwards.  A coarse multirate step captured while the
 * timers are on runs its levels one after another on one stream (without
 * them each level runs on its own branch, the levels overlapping), so every
 * timed launch has the GPU to itself and its time is that kernel's alone. */
fc_status fc_timers_enable(fc_forest* forest, int enable);

/* CUDA-graph replay of fc_step_multirate (on by default).  The first coarse
 * step for a given layout, dt_coarse and buffer parity is captured into a
 * graph (on an internal stream) and launched; later steps with the same key
 * replay it after writing their start time to device memory, so a step costs
 * two launches on `stream`.  A regrid discards the captured steps.  With
 * timers on, a replayed graph re-records its own events: read the timers
 * after each step to accumulate every step.  enable = 0 reverts to direct
 * launches (same kernels, same results). */
fc_status fc_set_graphs(fc_forest* forest, int enable);

/* Patch-update kernel variants: 0 "staged" (one CTA per patch, the whole
 * tile in shared memory, every thread on every phase -- low latency for
 * launches of few patches), 1 "walk" (lanes own patch columns and walk
 * the rows with warp shuffles, tiles double-buffered per warp by TMA, a
 * persistent grid of `warps`-warp CTAs -- fewest instructions per cell),
 * 2 (walk1: the walk with one tile buffer per warp, twice the warps per SM)
 * and 3 "band" (one CTA of `warps` warps per patch, each warp walking a band
 * of rows as the walk does: mx^2 / (32 warps) rows a band, at least one;
 * with refluxing and the cubed sphere's capacity form).  Where the walk
 * lacks what the forest needs (refluxing, the capacity form) the launch
 * runs staged.
 *
 * Untuned launch sizes run walk from 1024 patches up on planar grids, band
 * with 8 warps otherwise.
 *
 * fc_autotune times every candidate (staged; band with 4 or 8 warps;
 * walk with 2, 4, 8 warps per
 * CTA; walk1 with 4 or 8; each with the level's ghosts filled inside the update kernel or by
 * separate fill kernels) as a whole level substep of the current layout,
 * eight substeps replayed from one CUDA graph as in a captured step (walk
 * only for launches of at least two patches per SM: below that staged has
 * measured about twice as fast), and keeps the fastest per launch size (sizes bucketed by powers of two; a
 * bucket is tuned once per forest).  It overwrites the previous-state
 * buffers, so call it when all levels hold the same time (after set_q or a
 * regrid).  report: host, nullable, 32 x 4 ints per bucket b (patches in
 * [2^b, 2^(b+1))): (variant or -1 if untuned, warps, fused, ns per substep).
 * Synchronous.
 *
 * fc_set_advance_variant forces a variant for every launch (variant -1
 * restores the tuned/heuristic choice); warps is 2, 4 or 8, or 16 for band
 * (FC_ERR_INVALID_ARG otherwise). */
fc_status fc_autotune(fc_forest* forest, int* report, void* stream);

/* Fused ghost fill in multirate substeps (on by default): the patch-update
 * kernel applies Alg. 1 to the ghost ring of the tile it holds in shared
 * memory, so a level substep is one fill launch (the coarse neighbours'
 * time-interpolated data) plus the update, and the level's ghost cells are
 * never written to HBM.  enable = 0: separate fill kernels write every ghost
 * ring first (same results, bit for bit). */
fc_status fc_set_fused_fill(fc_forest* forest, int enable);
fc_status fc_set_advance_variant(fc_forest* forest, int variant, int warps);

/* Launch limits (tests and tuning).
 *   walk_ctas   cap on the persistent walk grid (0: as many CTAs as the SMs
 *               hold at once); a small cap makes every warp loop over many
 *               groups of patches through both of its tile buffers.
 *   wait_polls  polls of the patch-update kernels' bounded wait for their
 *               tile copies before they give up (negative: the default,
 *               2^22); 0 makes every such wait give up at once.  A kernel
 *               that gives up sets the forest's device error word (the next
 *               synchronising call returns FC_ERR_TIMEOUT and clears it),
 *               still waits, with the default limit, for the copies it has
 *               in flight, and leaves its patches not updated.
 * Captured steps are discarded (they carry the old values). */
fc_status fc_set_limits(fc_forest* forest, int walk_ctas, int64_t wait_polls);
fc_status fc_timers_read(fc_forest* forest, int phase, double* ms, int64_t* launches,
                         double* bytes, int reset);

/* Interior cell capacities in field order, nleaves x mx x mx doubles: h^2 on
 * the square domains (h = 2^-level / mx), the spherical cell area kappa on the
 * cubed sphere (Sec. 5.3 mapped grids; the FP64 metric the update uses).
 *   on_device  nonzero: `out` is a device pointer (async on `stream`);
 *              zero: a host pointer (the call synchronises `stream`). */
fc_status fc_forest_get_capacity(const fc_forest* forest, double* out, int on_device,
                                 void* stream);

/* Mass sums without any allocation.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they need the sum (an allocator
 * callback, a runtime that owns the device memory, a loop that must not
 * touch the allocator).  It computes the same per-forest FP64 mass as
 * fc_forest_mass, from a field the caller already holds, and keeps its
 * per-leaf partial sums in a fixed device array of FC_NOALLOC_MAX_LEAVES
 * doubles that every GPU loading this library holds until the process
 * exits.  It calls no cudaMalloc/cudaFree and no allocating library routine.
 *
 *   q             device, packed interior field [leaf][j][i] of `dtype`
 *                 (FC_F32 / FC_F64), mx x mx cells per leaf.
 *   capacity      device, nullable: the cells' capacities in the same
 *                 layout (doubles, as fc_forest_get_capacity returns them).
 *                 Null: each cell weighs h^2, h = 2^-level / mx (the square
 *                 domains; the same bits as fc_forest_mass there).  Given:
 *                 each cell weighs its capacity (on the cubed sphere the
 *                 same bits as fc_forest_mass, which sums kappa q).
 *   level         device, nleaves ints: refinement level of each leaf.
 *   forest_start  device, nforests+1 ints with 0 = forest_start[0] <= ... <=
 *                 forest_start[nforests] = nleaves: the leaves of forest f
 *                 are [forest_start[f], forest_start[f+1]) in the field
 *                 order.  Entries outside that contract are clamped into
 *                 [0, nleaves] on the device (the sums are then of the
 *                 clamped ranges); no slot outside this call's leaves is read.
 *   out           device, nforests doubles: each leaf is summed in a fixed
 *                 order, then the leaves of a forest in a fixed order.
 * nleaves above FC_NOALLOC_MAX_LEAVES is rejected (FC_ERR_INVALID_ARG).
 * Work is enqueued on `stream`; the call does not synchronise.  All calls
 * share the one array: calls whose work overlaps on the GPU (other streams,
 * other threads) race and must be serialised by the caller.  The first call
 * on a device looks up the array's device address with that device current
 * and keeps it for the life of the process; make that first call before any
 * stream capture, and do not use the call after cudaDeviceReset (or any
 * other teardown of the device's primary context) in the same process. */
#define FC_NOALLOC_MAX_LEAVES (1 << 19)
fc_status fc_mass_noalloc(const void* q, const double* capacity, int dtype, int mx, int nleaves,
                          const int* level, const int* forest_start, int nforests, double* out,
                          void* stream);

/* Thread-local description of the last failure. */
const char* fc_last_error(void);

/* Kernel launches issued by this thread since the last reset. */
uint64_t fc_launch_count(int reset);

#ifdef __cplusplus
}
#endif
#endif /* FC_H */
