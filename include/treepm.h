/*
 * treepm.h -- C ABI of libtreepm, a GB300 (sm_103a) implementation of the
 * TreePM gravitational force on the currently active particles, as described
 * in Weinberger, Springel & Pakmor, "The AREPO public code release"
 * (Sec. 3 gravity, Sec. 7.1-7.3 time stepping).
 *
 * The library builds an oct-tree with monopole moments for a particle set
 * (Sec. 3.1), keeps it resident on the GPU, and evaluates the force and
 * potential on any subset of "active" particles from the full mass
 * distribution (Sec. 7.3: an active particle interacts with all mass).  The
 * force may be split into a short-range tree part and a long-range
 * particle-mesh part (Sec. 3.3, 3.4): always for a periodic box, optionally
 * for open boundaries (zero-padded mesh).  Around the force path, drift,
 * due-set and kick calls step a system through a power-of-two time-bin
 * hierarchy (Sec. 7.1-7.3).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every call returns a tpm_status.  Nothing is thrown and nothing aborts
 *   across the ABI.  tpm_last_error() gives a message for the last failing
 *   call of the calling thread.
 * - Pointers may be host or device memory; the library tells them apart with
 *   cudaPointerGetAttributes.  Device pointers must belong to the context's
 *   device.  With host pointers a call copies inputs in, runs, copies results
 *   out and synchronises the stream before returning, except that the tree
 *   build reads page-locked host inputs (cudaHostAlloc, cudaHostRegister) in
 *   place through their mapped device address (the CPU-GPU link is coherent
 *   on this platform); with device pointers a call is stream-ordered on
 *   `stream` (a cudaStream_t, NULL = legacy default stream) and returns once
 *   the work is enqueued (the tree build itself synchronises `stream` once,
 *   to read the node count, after its last read of the inputs).
 * - The caller owns every buffer it passes.  Inputs are read during the call
 *   (host) or before the stream reaches the end of the call's work (device)
 *   and may be reused afterwards.  The library owns the resident trees and
 *   all of its scratch memory, drawn from a per-context pool under the HBM
 *   budget given at tpm_create.
 * - Arrays are tightly packed, C order: positions are n x 3 doubles
 *   (x, y, z per particle), accelerations n_active x 3 floats.
 * - Units are set by G; the library applies no other scaling.
 */
#ifndef TREEPM_H
#define TREEPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TPM_API_VERSION 2

typedef struct tpm_ctx tpm_ctx; /* opaque: device, memory pool, resident systems */
typedef uint64_t tpm_sys;       /* handle of a resident particle system; 0 is never valid */

typedef enum {
    TPM_OK = 0,
    TPM_EINVAL = -1,           /* malformed argument (null pointer, bad size, bad parameter) */
    TPM_EBUDGET = -2,          /* admission refused: the call would exceed the HBM budget; no side effects */
    TPM_ENOSYS_HANDLE = -3,    /* unknown or released system handle */
    TPM_ECUDA = -4,            /* a CUDA runtime / cuFFT call failed; the message names it */
    TPM_ETIMEDOUT = -5,        /* reserved: no kernel of this library waits on another block or on a
                                  flag, so no call returns it */
    TPM_ENAN = -6              /* non-finite input (position, mass, |a_old|) */
} tpm_status;

typedef enum {
    TPM_CRIT_BH = 0,       /* geometric criterion: open if L > theta d (Sec. 3.1) */
    TPM_CRIT_RELATIVE = 1  /* relative criterion: open if G M L^2 / d^4 > alpha |a_old| (Sec. 3.1) */
} tpm_crit;

/* Parameters of a tree build (Sec. 3.1, 3.2). */
typedef struct {
    double G;            /* gravitational constant, > 0 */
    double h;            /* spline softening support, > 0: Newtonian beyond h; h = 2.8 eps (Sec. 3.2) */
    int32_t periodic;    /* 0: open boundaries; 1: periodic cube [0, box)^3 */
    double box;          /* periodic box side (> 0; ignored when periodic = 0) */
    double shift[3];     /* random root placement in [0, 1)^3 drawn by the caller per build
                            (Sec. 3.1: randomised tree domain / random box shift) */
    int32_t leaf_bucket; /* B >= 1: a cell holding more than B particles is split; B = 1 is the paper's tree */
} tpm_build_params;

/* Parameters of a force evaluation (Sec. 3.1, 3.4; names of Table 1). */
typedef struct {
    int32_t crit;       /* tpm_crit */
    double theta;       /* ErrTolTheta, used when crit = TPM_CRIT_BH (> 0) */
    double alpha;       /* ErrTolForceAcc, used when crit = TPM_CRIT_RELATIVE (>= 0) */
    int32_t box_guard;  /* 1: always open a node whose 1.2 L cube around its centre holds the particle */
    int32_t treepm;     /* 1: short-range tree force + long-range PM (open systems: the zero-padded isolated
                           mesh); 0 on a periodic system: the tree with the Ewald correction */
    int32_t pm_n;       /* PMGRID: mesh points per side (power of two, 8..1024) */
    double asmth;       /* ASMTH a_s: split scale r_s = a_s box / pm_n */
    double rcut;        /* RCUT a_cut: tree cutoff radius a_cut r_s */
    int32_t pm_grad;    /* mesh force of a periodic system (Sec. 3.3 leaves the stencil open):
                           TPM_GRAD_FD4 (0) the 4-point finite difference of the potential mesh,
                           TPM_GRAD_IK (1) the spectral derivative -i k Phi_k (three more inverse
                           transforms, three force meshes kept with the system) */
    int32_t plain_fp32; /* 0: mixed precision (offsets from each walk group's frame taken in FP64, pair math
                           in FP32); 1 (open boundaries; a comparison arm, not a recommendation): the plain
                           FP32 form, every pair vector a difference of absolute FP32 coordinates, as a
                           code that holds its positions in FP32 computes it */
} tpm_force_params;

#define TPM_GRAD_FD4 0
#define TPM_GRAD_IK 1

/* Version of this header the library was built from (TPM_API_VERSION). */
int tpm_version(void);

/* Process-wide counts since the library was loaded: launches of the
 * library's own kernels, and calls of CUB device primitives (radix sort,
 * scan), each of which launches a few kernels of its own.  Either pointer
 * may be NULL. */
int tpm_launch_counts(uint64_t *kernels, uint64_t *cub_calls);

/* Message for the last failing call on the calling thread ("" if none).
 * The pointer stays valid until the thread's next library call. */
const char *tpm_last_error(void);

/* Creates a context on CUDA device `device` whose allocations (trees, meshes,
 * scratch) may total at most `hbm_budget_bytes` (0 = 90% of the free memory).
 * *ctx receives the context.  Errors: TPM_EINVAL (null ctx, bad device),
 * TPM_ECUDA. */
int tpm_create(tpm_ctx **ctx, int device, size_t hbm_budget_bytes);

/* Releases every system of the context and the context itself.  Waits for the
 * context's outstanding work.  A null ctx is a no-op. */
int tpm_destroy(tpm_ctx *ctx);

/* Bytes currently held by resident systems and the budget. */
int tpm_memory(const tpm_ctx *ctx, size_t *used_bytes, size_t *budget_bytes);

/*
 * Builds the oct-tree of n particles and keeps it resident (Sec. 3.1):
 * cubic root of power-of-two side L0 (open boundaries: the smallest with
 * L0 >= 1.25 x the largest extent, placed at lo - shift (L0 - extent) on the
 * 2^-21 L0 grid; periodic: [0, box) after shifting all positions by
 * shift x box and wrapping), 63-bit Morton keys of the 21-bit cell
 * coordinates, a stable (key, index) sort, the cells of every level that hold
 * particles and whose parent holds more than B, and FP64 masses and centres
 * of mass summed children-first in ascending octant order.  The tree is
 * rebuilt from scratch for every call, as in the paper (one build per local
 * step).
 *   pos   n x 3 positions (FP64).  Periodic positions must lie in [0, box).
 *   mass  n masses (FP32, > 0).
 *   out   receives the system handle.
 * Errors: TPM_EINVAL (n < 1, n > 2^31 - 1, bad params), TPM_ENAN (non-finite
 * position or mass), TPM_EBUDGET, TPM_ECUDA.
 */
int tpm_build_tree(tpm_ctx *ctx, const double *pos, const float *mass, int64_t n, const tpm_build_params *p,
                   void *stream, tpm_sys *out);

/*
 * tpm_build_tree with per-particle softening (Sec. 3.2): hsoft holds each
 * particle's spline support (n FP32 > 0, host or device; p->h is then not
 * used by the walk).  A pair interacts with the larger of its two supports;
 * an accepted node with the larger of the target's support and the node's
 * largest; a node holding particles of different supports is always opened
 * for a target whose support is smaller than the node's largest and whose
 * distance to the node's centre of mass is below that largest.  Open
 * boundaries only (with or without treepm).  The node set and monopoles are
 * those of tpm_build_tree.  Errors: as tpm_build_tree, TPM_EINVAL (null
 * hsoft, periodic system), TPM_ENAN (a support not finite or not > 0).
 */
int tpm_build_tree_soft(tpm_ctx *ctx, const double *pos, const float *mass, const float *hsoft, int64_t n,
                        const tpm_build_params *p, void *stream, tpm_sys *out);

/*
 * Long-range particle-mesh potential (Sec. 3.3, 3.4), r_s = asmth dx.
 * Periodic systems: CIC assignment of all mass onto pm_n^3 mesh points at
 * x = i dx, dx = box / pm_n, FFT, multiplication by -4 pi G / k^2
 * exp(-k^2 r_s^2) / W(k)^2 with the CIC window W = prod_a sinc^2(k_a dx / 2)
 * and the k = 0 mode removed (mean density subtracted), inverse FFT.
 * Open boundaries (zero padding and the isolated Green's function): pm_n^3
 * mesh points over a cube of the tree root's side L0 centred on the particles'
 * bounding box (dx = L0 / pm_n), inside a zero-padded (2 pm_n)^3 mesh; the
 * potential is the convolution of the CIC masses with the long-range kernel
 * -G erf(r / 2 r_s) / r sampled at the padded mesh's circular separations,
 * divided by W(k)^2 in k-space, k = 0 kept (pm_n <= 512).  The mesh force is
 * the 4-point finite difference of the potential mesh, or for a periodic
 * system with pm_grad = TPM_GRAD_IK the spectral derivative: a_k = -i k_a
 * Phi_k per axis (the Nyquist mode of each axis set to zero), three more
 * inverse transforms into three force meshes.  The meshes stay with the
 * system until the next call or release; tpm_compute_forces with treepm = 1
 * interpolates from them (the call's pm_grad must match).  Errors: TPM_EINVAL
 * (treepm = 0, bad pm_n / asmth / rcut / pm_grad, pm_grad = TPM_GRAD_IK on
 * an open system), TPM_ENOSYS_HANDLE, TPM_EBUDGET, TPM_ECUDA.
 */
int tpm_pm_long_range(tpm_ctx *ctx, tpm_sys s, const tpm_force_params *p, void *stream);

/*
 * Gravitational acceleration and potential on active particles (Sec. 3.1-3.4).
 * Each active particle walks the tree from the root: with treepm, a node whose
 * cube lies farther than a_cut r_s is skipped; a node is opened when the
 * particle lies in the 1.2 L cube around the node centre (box_guard) or the
 * criterion asks for it; an opened internal node hands over to its children,
 * an opened leaf interacts particle by particle (never with the particle
 * itself), and an unopened node contributes its monopole.  The pair law is
 * the spline-softened Newtonian force (Sec. 3.2), times the short-range
 * factor erfc(r/2r_s) + r/(sqrt(pi) r_s) exp(-r^2/4r_s^2) under TreePM, to
 * which the mesh force (4-point finite differences, CIC interpolation) is then
 * added.  A periodic system with treepm = 0 is a pure tree with the Ewald
 * correction (Sec. 3.1): every term is taken at the nearest image and gets
 * the correction for all other images and the neutralising background,
 * interpolated trilinearly from a table of the Ewald sums over [0, box/2]^3
 * (65^3 points, built on the device once per context -- the first such call
 * allocates it), and each potential gets the particle's own lattice term.
 * Pair arithmetic is FP32 on positions taken relative to node and group
 * centres in FP64.
 *   active_ids  n_active indices into the particle order given at build time,
 *               or NULL for all particles in that order (n_active must be n).
 *               n_active = 0 returns TPM_OK at once (the arrays may be NULL).
 *   a_old       n_active |a| from the previous evaluation (relative criterion),
 *               or NULL (only with TPM_CRIT_BH).
 *   acc         out: n_active x 3 accelerations, in active_ids order.
 *   pot         out: n_active potentials (may be NULL).  Periodic potentials
 *               are defined up to a constant.
 *   n_int       out: n_active particle-node + particle-particle interaction
 *               counts (may be NULL): the cost factor g_i of Sec. 8.
 * Errors: TPM_EINVAL, TPM_ENOSYS_HANDLE, TPM_ENAN (non-finite a_old),
 * TPM_EBUDGET, TPM_ECUDA.
 */
int tpm_compute_forces(tpm_ctx *ctx, tpm_sys s, const uint32_t *active_ids, int64_t n_active, const float *a_old,
                       const tpm_force_params *p, float *acc, float *pot, uint32_t *n_int, void *stream);

/*
 * tpm_compute_forces without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot let a library
 * allocate device memory inside their time-step loop -- programs that have
 * already given the device memory to their own allocator, or that must not
 * pay for (or risk failing) an allocation at every step.  The per-call
 * scratch of tpm_compute_forces (the active set sorted into key order and
 * the sort's temporary storage) lives instead in one fixed-size device array
 * inside the library, about 8 MiB, which every GPU that loads the library
 * holds until the process exits.
 *   Same arguments and results as tpm_compute_forces, except:
 *   - active_ids is required and n_active must lie in [1, TPM_NOALLOC_MAX_ACTIVE];
 *     larger sets are rejected with TPM_EINVAL;
 *   - every array (active_ids, a_old, acc, pot, n_int) must be device memory
 *     of the context's GPU (host arrays would need staging buffers):
 *     TPM_EINVAL otherwise;
 *   - ids are not checked on the host: an id >= n is read as particle 0 and
 *     sets the system's status word, which the next tpm_sync_status reports
 *     as TPM_EINVAL (as for device ids given to tpm_compute_forces);
 *   - the call is stream-ordered and never synchronises;
 *   - on a periodic system without treepm the context's Ewald table must
 *     exist already (any tpm_compute_forces call of that kind builds it):
 *     TPM_EINVAL otherwise.
 * The first call on a device looks up the array's device address (it loads
 * the library's device code on that device), so make that first call before
 * any stream capture.  All calls share the one array, which keeps the last
 * call's contents: two calls whose work overlaps on the GPU (different
 * streams, or different contexts on one device) race on it and must be
 * ordered by the caller.
 */
#define TPM_NOALLOC_MAX_ACTIVE (1 << 18)
int tpm_compute_forces_noalloc(tpm_ctx *ctx, tpm_sys s, const uint32_t *active_ids, int64_t n_active,
                               const float *a_old, const tpm_force_params *p, float *acc, float *pot,
                               uint32_t *n_int, void *stream);

/*
 * Batched evaluation (hierarchical time-step batching, serving).  The paper
 * integrates with local power-of-two time steps (Sec. 7.2): each substep
 * evaluates forces only for the particles of the active time bins, from the
 * full mass distribution (Sec. 7.3); a force server likewise sees many small
 * requests.  A plan holds all the scratch of a batch, so a batched call only
 * enqueues device work -- no allocation, no host synchronisation -- and a
 * sequence of batched calls can be captured in a CUDA graph.  All requests
 * of one call run in one persistent walk launch: resident warps take groups
 * of at most G consecutive (key-ordered) particles of any request from a
 * device work queue.  Open-boundary systems only.
 */
typedef struct tpm_plan tpm_plan;

/* Flag: each request's ids are already in the key order of its tree (as
 * produced by cutting an active set sorted by tree rank); skips the sort. */
#define TPM_BATCH_PRESORTED 1u

/* Creates a plan for batches of at most max_ids ids in max_requests
 * requests (memory drawn from ctx's budget: about 40 B per id + 300 B per
 * request).  Errors: TPM_EINVAL, TPM_EBUDGET, TPM_ECUDA. */
int tpm_plan_create(tpm_ctx *ctx, int64_t max_ids, int64_t max_requests, tpm_plan **plan);

/* Frees a plan (waits for the device). */
int tpm_plan_destroy(tpm_ctx *ctx, tpm_plan *plan);

/* Walk group size G in [8, 32] (one particle per lane of a warp) or 64 (two
 * particles per lane: each node record the warp reads serves 64 particles),
 * default 32, and its current value. */
int tpm_plan_set_group_size(tpm_plan *plan, int group_size);
int tpm_plan_group_size(const tpm_plan *plan);

/* Capacity of the batched walk's per-warp candidate stack: 128, 192
 * (default) or 256 entries (a deeper stack takes more shared memory per warp;
 * above capacity - 64 entries the walk takes one candidate at a time), and its
 * current value.  Errors: TPM_EINVAL for other values. */
int tpm_plan_set_stack_depth(tpm_plan *plan, int depth);
int tpm_plan_stack_depth(const tpm_plan *plan);

/*
 * Forces for n_req requests in one launch.  Request r evaluates
 * tpm_compute_forces for system systems[r] with params[r] on the ids
 * ids[offsets[r] .. offsets[r+1]) (offsets: host array of n_req + 1, starting
 * at 0, non-decreasing).  ids, a_old (per id, required if any request uses the
 * relative criterion), acc (3 per id), pot and n_int (per id, may be NULL) are
 * DEVICE arrays indexed by position in ids.  systems and params are host
 * arrays; they are copied into the plan during the call.  Stream-ordered;
 * never synchronises except to wait until the previous call on the plan has
 * copied its host arguments (skipped while `stream` is being captured).
 * Device-side errors (out-of-range ids) surface in tpm_plan_sync_status.
 * Errors: TPM_EINVAL (sizes beyond the plan, periodic systems, host arrays),
 * TPM_ENOSYS_HANDLE, TPM_ECUDA.
 */
int tpm_compute_forces_batch(tpm_ctx *ctx, tpm_plan *plan, int64_t n_req, const tpm_sys *systems,
                             const int64_t *offsets, const tpm_force_params *params, const uint32_t *ids,
                             const float *a_old, float *acc, float *pot, uint32_t *n_int, uint32_t flags,
                             void *stream);

/* Waits for `stream`; reports and clears device-side errors of the plan's
 * batches (TPM_EINVAL: an id out of range; TPM_ECUDA: walk stack overflow). */
int tpm_plan_sync_status(tpm_ctx *ctx, tpm_plan *plan, void *stream);

/* Times the batch for G in {8, 16, 32, 64} x stack depth in {128, 192, 256}
 * (reps timed runs each, after one warm-up), keeps the fastest pair in the
 * plan and returns its G (read the depth with tpm_plan_stack_depth) with its
 * median time in milliseconds.  Synchronises.  Arguments as
 * tpm_compute_forces_batch. */
int tpm_plan_autotune(tpm_ctx *ctx, tpm_plan *plan, int64_t n_req, const tpm_sys *systems, const int64_t *offsets,
                      const tpm_force_params *params, const uint32_t *ids, const float *a_old, float *acc,
                      float *pot, uint32_t *n_int, uint32_t flags, int reps, void *stream, int *best_group,
                      float *best_ms);

/* Waits for `stream` and reports errors that device work recorded for system
 * s since the last check (then clears them): TPM_EINVAL if a device-side
 * active id was out of range (its outputs hold particle 0's values), TPM_ECUDA
 * if the walk's candidate stack overflowed; TPM_OK otherwise. */
int tpm_sync_status(tpm_ctx *ctx, tpm_sys s, void *stream);

/* FP64 conservation diagnostics of forces on all n particles of system s
 * (the momentum and energy checks of a gravity solver, Sec. 7).  acc (n x 3
 * FP32), pot (n FP32, may be NULL) and vel (n x 3 FP64, may be NULL) are
 * DEVICE arrays in the caller's particle order; the masses are the system's.
 * out (host, 9 doubles): [0..2] total force sum_i m_i a_i (zero for an
 * exactly symmetric interaction; a tree leaves a residual of the size of its
 * force errors), [3] potential energy 1/2 sum_i m_i phi_i (0 without pot),
 * [4] kinetic energy 1/2 sum_i m_i |v_i|^2 and [5..7] momentum sum_i m_i v_i
 * (0 without vel), [8] sum_i m_i |a_i|, the scale of [0..2].  FP64 sums in a
 * fixed order (the same bits on every run on the same GPU model).
 * Synchronises.  Errors: TPM_EINVAL (null or host arrays), TPM_ENOSYS_HANDLE,
 * TPM_ECUDA. */
int tpm_diagnostics(tpm_ctx *ctx, tpm_sys s, const float *acc, const float *pot, const double *vel, double *out,
                    void *stream);

/* Frees a resident system.  Waits for its outstanding work. */
int tpm_release(tpm_ctx *ctx, tpm_sys s);

/* Size and root of a resident system: particle count, node count, root corner
 * x0[3] and side L0 (periodic: x0 = 0, L0 = box). */
int tpm_tree_info(tpm_ctx *ctx, tpm_sys s, int64_t *n, int64_t *n_nodes, double *x0, double *L0);

/*
 * Host copies of a resident tree, for checking (synchronous).  Any pointer may
 * be NULL.  Particle arrays have n entries in sorted order: key (Morton key of
 * the 21-bit cell coordinates, x in bit 0, y bit 1, z bit 2 of each triplet),
 * perm (original index).  Node arrays have n_nodes entries in depth-first
 * pre-order (children in ascending octant): level, prefix (key >> 3 (21 -
 * level)), first sorted particle, particle count, skip (index of the first
 * node after the subtree), FP64 mass and centre of mass (n_nodes x 3).
 * xtree (n x 3, original order) receives the positions the tree uses (after
 * the periodic shift and wrap).
 */
int tpm_tree_export(tpm_ctx *ctx, tpm_sys s, uint64_t *key, uint32_t *perm, uint8_t *level, uint64_t *prefix,
                    uint32_t *first, uint32_t *count, uint32_t *skip, double *mass, double *com, double *xtree);

/* Host copy of the long-range mesh potential of the last tpm_pm_long_range on
 * s: m^3 floats, C order x, y, z, with m = pm_n (periodic) or 2 pm_n (open
 * boundaries: the zero-padded mesh, physical for indices <= pm_n).
 * count must be m^3.  Synchronous. */
int tpm_pm_export(tpm_ctx *ctx, tpm_sys s, float *phi, int64_t count);

/* ---------------------------------------------------------------------------
 * Time stepping around the force path (Sec. 7.1-7.3).
 *
 * A cycle of length T is cut into 2^N ticks of dt_tick = T / 2^N
 * (N = nbins - 1).  Bin b (0 <= b <= N) has the step dt_tick 2^(N - b): bin 0
 * is the longest step, bin N the shortest.  Bin b is due at tick t (taken
 * modulo 2^N) when t is a multiple of 2^(N - b).  A particle's step may not
 * exceed sqrt(2 C_grav eps / |a|) (Sec. 7.1; the paper prints the inequality
 * reversed, an upper bound is meant); it takes the bin of the largest step
 * not above that.  Moving to a shorter step is always allowed, to a longer
 * one only onto a bin that is due at the current tick (Sec. 7.2): a particle
 * asking for a longer step that is not due takes the longest due step
 * between the one it asks for and its current one.  Kick-drift-kick leapfrog
 * (Sec. 7.3): each step opens and closes with a half kick v += a dt / 2, all
 * particles drift every tick, and the tree is rebuilt at every tick for the
 * forces on the particles due.  FP64 positions and velocities; every FP64
 * update uses round-to-nearest multiplies and adds in a fixed order.
 * --------------------------------------------------------------------------- */
typedef struct {
    double dt_tick; /* the shortest step, T / 2^(nbins - 1) (> 0) */
    int32_t nbins;  /* number of bins, 1..31 */
    double c_grav;  /* ErrTolIntAccuracy C_grav (> 0) */
    double eps;     /* softening length of the criterion (> 0; eps = h / 2.8) */
} tpm_step_params;

/*
 * Drift: x += v dt for n particles (pos, vel: n x 3 FP64, device memory).
 * With periodic = 1 every coordinate is wrapped back into [0, box).
 * Errors: TPM_EINVAL (null pointers, host memory, n < 0, non-finite dt,
 * box <= 0 when periodic), TPM_ECUDA.
 */
int tpm_drift(tpm_ctx *ctx, double *pos, const double *vel, int64_t n, double dt, int32_t periodic, double box,
              void *stream);

/*
 * The particles due at `tick`: their indices, ascending, into ids (device,
 * room for n), and their number into *n_active (host; the call waits for the
 * stream).  With a_old non-NULL, a_old[k] = amag[ids[k]] (device arrays) --
 * the |a| of the previous force evaluation that the relative criterion needs.
 *   bins  n time bins (int8, device), as written by tpm_kick.
 * Errors: TPM_EINVAL (null pointers, host memory, n outside [1, 2^31 - 1],
 * nbins outside [1, 31], tick < 0), TPM_EBUDGET (scratch), TPM_ECUDA.
 */
int tpm_active_set(tpm_ctx *ctx, const int8_t *bins, const float *amag, int64_t n, int64_t tick, int32_t nbins,
                   uint32_t *ids, float *a_old, int64_t *n_active, void *stream);

/*
 * Kicks for the n_active particles ids[k] (< n; others are skipped) whose
 * accelerations acc[k] (n_active x 3 FP32, in ids order) were just computed
 * at `tick`: the closing half kick with the step of the particle's current
 * bin (skipped when first = 1, the start of the integration), the new bin
 * from the step criterion and the nesting rule (with first = 1 any bin may
 * be taken), the opening half kick with the new step, and amag[i] = |a|
 * (FP32) for the next relative criterion.  vel (n x 3 FP64), bins (n int8),
 * amag (n FP32): device memory, updated in place.
 * Errors: TPM_EINVAL (null pointers, host memory, bad params), TPM_ECUDA.
 */
int tpm_kick(tpm_ctx *ctx, const uint32_t *ids, int64_t n_active, int64_t n, const float *acc, double *vel,
             int8_t *bins, float *amag, int64_t tick, const tpm_step_params *p, int32_t first, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TREEPM_H */
