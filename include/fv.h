/*
 * fv.h -- C ABI of the batched finite-volume patch library (libfv.so).
 *
 * The library advances many small Cartesian patches of a block-structured
 * mesh by one explicit Euler step of a Rusanov finite-volume scheme for the
 * compressible Euler equations, as in arXiv 2302.09005 ("GPU Offloading in
 * ExaHyPE Through C++ Standard Algorithms"):
 *   - PDE and flux f^j(q): Sec. 2, Eq. 1-2 (energy flux (E+p) j_j / rho);
 *   - update Q^{n+1} = Q^n - dt/dx sum_j (F_{+1/2} - F_{-1/2}): Eq. 3,
 *     Algorithm 1 step 7;
 *   - Rusanov face flux F = 1/2 [f(Q_L) + f(Q_R) - a (Q_R - Q_L)]: Eq. 4;
 *   - a = max over the two states of |u_j| + c: Eq. 5;
 *   - per-patch maximum eigenvalue: Algorithm 1 step 10;
 *   - a batch of N patches in one kernel invocation: Sec. 3 (batched kernel).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Device pointers.  Every array argument is a DEVICE pointer owned by the
 * caller (for example the data pointer of a CUDA tensor), unless its
 * description says "host".  The library never frees caller memory.
 *
 * Asynchrony.  Every call that launches work enqueues it on the handle's
 * CUDA stream and returns without synchronising.  Arguments are validated on
 * the host before anything is enqueued; an invalid call enqueues nothing and
 * returns an error status.  Per-patch metadata lives on the device and is
 * checked by the kernels: a patch with an invalid size or offset is skipped
 * and flags the handle's device status word (read it with fv_get_status).
 *
 * Patch layout.  Patch i occupies the elements
 *   [patch_offsets[i], patch_offsets[i] + (p_i + 2h)^d * s)
 * of a flat buffer of doubles (FV_FP64 handles) or floats (FV_FP32 handles),
 * with p_i = patch_sizes[i] interior cells per axis and halo width h.  Cells
 * are ordered x fastest, then y, then z; the s unknowns of a cell are
 * contiguous: (rho, j_1, .., j_d, E) with j = rho u the momentum and E the
 * total energy.  Interior cells have every coordinate in [h, h+p_i).
 * Every offset must be a multiple of 16 bytes (2 doubles / 4 floats).
 *
 * Errors.  Functions return fv_status.  FV_ERR_CUDA carries the CUDA error
 * text in fv_last_error().  No entry point traps or aborts the process.
 */
#ifndef FV_H
#define FV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FV_OK = 0,
  FV_ERR_INVALID_ARG = 1, /* bad argument; nothing was enqueued            */
  FV_ERR_ALIGNMENT = 2,   /* a pointer or patch offset is not 16-B aligned */
  FV_ERR_UNSUPPORTED = 3, /* valid but not supported (d, s, p, halo)       */
  FV_ERR_CUDA = 4,        /* a CUDA call failed; see fv_last_error         */
  FV_ERR_NONPHYSICAL = 5, /* a kernel met rho <= 0, p <= 0 or a NaN        */
  FV_ERR_TIMEOUT = 6,     /* a bounded device wait gave up                 */
  FV_ERR_BAD_PATCH = 7    /* a kernel skipped a patch with bad metadata    */
} fv_status;

typedef enum {
  FV_FP64 = 0, /* buffers of double, all arithmetic in FP64 */
  FV_FP32 = 1  /* buffers of float, flux and update arithmetic in FP32;
                  maximum reductions, dt and conservation sums in FP64 */
} fv_precision;

typedef struct {
  double gamma;           /* ratio of specific heats, > 1 (1.4 for air)      */
  int halo;               /* halo width h; the Rusanov update needs 1        */
  fv_precision precision; /* element type of every buffer of this handle    */
  int max_patch_size;     /* largest p the handle will be given; bounds the
                             shared memory of the update kernel.  0 selects
                             8 for d = 3 and 17 for d = 1, 2.                 */
} fv_options;

/* Fills *o with gamma = 1.4, halo = 1, FV_FP64, max_patch_size = 0. */
void fv_options_default(fv_options* o);

typedef struct fv_batch fv_batch; /* opaque handle */

/*
 * fv_batch_create -- make a handle for d-dimensional patches with s unknowns
 * per cell (the Euler system has s = d + 2, Sec. 2), options o (NULL for the
 * defaults) and the CUDA stream cuda_stream (a cudaStream_t; NULL is the
 * legacy default stream) on the current CUDA device.
 * The handle allocates its own small device workspace (status word, time
 * step slot, reduction partials).  d in {1, 2, 3}; s == d + 2.
 * Returns FV_ERR_INVALID_ARG for a bad d, s or option, FV_ERR_CUDA if the
 * workspace cannot be allocated.  *out is NULL on error.
 */
fv_status fv_batch_create(fv_batch** out, int d, int s, const fv_options* o, void* cuda_stream);

/* Releases the handle and its workspace (synchronises its stream first). */
fv_status fv_batch_destroy(fv_batch* h);

/* Makes later calls enqueue on cuda_stream. */
fv_status fv_batch_set_stream(fv_batch* h, void* cuda_stream);

/*
 * fv_patch_update_batch -- one explicit Euler step (Eq. 3) of n_patches
 * patches with Rusanov face fluxes (Eq. 4-5): Algorithm 1 with the outer
 * loop over patches, every face flux computed once and used by both cells.
 *   in_with_halo  device, patches at Q^n with filled halos; read only.
 *   out           device, same layout; the interior cells of every patch are
 *                 overwritten with Q^{n+1}; its halo cells are not written.
 *                 Must not overlap in_with_halo.
 *   patch_offsets device int64[n_patches], element offsets into both buffers.
 *   patch_sizes   device int32[n_patches], p_i in [1, max_patch_size].
 *   d, s          must equal the handle's.
 *   dx            cell width (> 0), the same on every axis.
 *   dt            time step; dt <= 0 uses the device time step written by
 *                 the last fv_max_eigenvalue_reduce on this handle.
 * n_patches == 0 enqueues nothing and returns FV_OK.
 */
fv_status fv_patch_update_batch(fv_batch* h, const void* in_with_halo, void* out,
                                const int64_t* patch_offsets, const int32_t* patch_sizes,
                                int64_t n_patches, int d, int s, double dx, double dt);

/* Optional outputs and checks of fv_patch_update_batch_ex. */
typedef struct {
  double* lambda_patch; /* device double[n], per-patch max a over the faces
                           used (Algorithm 1 step 10), or NULL              */
  int64_t n_elems;      /* element count of both buffers; > 0 makes the
                           kernels skip (and flag) patches that would run
                           past it; 0 disables the check                    */
  const float* corr;    /* per-face flux corrections (2D handles; layout of
                           fv_flux_correction) added to F, or NULL          */
} fv_update_extras;

/* fv_patch_update_batch with optional outputs (extras may be NULL). */
fv_status fv_patch_update_batch_ex(fv_batch* h, const void* in_with_halo, void* out,
                                   const int64_t* patch_offsets, const int32_t* patch_sizes,
                                   int64_t n_patches, int d, int s, double dx, double dt,
                                   const fv_update_extras* extras);

/*
 * fv_halo_fill -- fills the face halo layers of every patch in place (the
 * engine's job of keeping halo data consistent, Sec. 2).  Edge and corner
 * halo cells are not touched; the Rusanov update does not read them.
 *   neighbours  device int32[n_patches * 2d], per patch in the order
 *               -x, +x, -y, +y, -z, +z:
 *                 >= 0 : index of the neighbouring patch, which must have the
 *                        same p; its h interior layers next to the shared
 *                        face are copied (a patch may be its own neighbour:
 *                        periodic);
 *                 -1   : outflow, each halo cell repeats the nearest
 *                        interior cell;
 *                 -2   : reflecting wall, mirror image of the interior with
 *                        the normal momentum negated.
 * The kernel reads only interior cells and writes only halo cells.  Patches
 * or neighbours with invalid metadata are skipped and flag the status word.
 */
fv_status fv_halo_fill(fv_batch* h, void* q_with_halo, const int64_t* patch_offsets,
                       const int32_t* patch_sizes, const int32_t* neighbours, int64_t n_patches);

/*
 * fv_max_eigenvalue_reduce -- per-patch and batch maximum wave speed and the
 * CFL time step (Eq. 5; Algorithm 1 step 10).
 * The per-patch value is the largest a = max(|u_j|+c of the two cells) over
 * the faces that bound interior cells -- the faces the update uses -- so it
 * equals the update's lambda_patch output on the same state.
 *   per_patch_max  device double[n_patches] or NULL.
 *   global_max     device double[1] or NULL: maximum over the batch (0 for
 *                  an empty batch).
 *   cfl, dx        > 0; dt = cfl * dx / (d * global max) is written to the
 *                  handle's device time step (read by an update with
 *                  dt <= 0) and to dt_out (device double[1]) if not NULL.
 * Maxima are exact, so the result does not depend on the order of work.
 * Uses the handle's workspace for per-block partial maxima.
 */
fv_status fv_max_eigenvalue_reduce(fv_batch* h, const void* q_with_halo,
                                   const int64_t* patch_offsets, const int32_t* patch_sizes,
                                   int64_t n_patches, double* per_patch_max, double* global_max,
                                   double cfl, double dx, double* dt_out);

/*
 * fv_patch_update_host -- fv_patch_update_batch on patches in HOST memory:
 * the paper's offload pattern (the engine ships a batch of patches with
 * their halos to the GPU for every update and takes the results back).  The
 * batch is cut into chunks of chunk_patches consecutive patches (<= 0: about
 * 256 MB per chunk); the copy in of a chunk, the update of the previous one
 * and the copy out of the one before overlap (two copy streams, the
 * handle's stream for the update, three device staging slots the handle keeps
 * until fv_batch_destroy).
 *   host_in, host_out  host buffers (pinned for overlap; pageable works,
 *                      slower), the layout of fv_patch_update_batch; the
 *                      interior cells of host_out receive Q^{n+1}, its halo
 *                      cells a copy of host_in's.  host_out == host_in
 *                      updates in place: then a chunk of equally spaced
 *                      patches of one size is copied in only from each
 *                      patch's first to its last face-halo cell (what the
 *                      update reads) and back only from its first to its
 *                      last interior cell, for 3D patches plane by plane
 *                      (each z-plane's cells (1, 1, z) .. (p, p, z): 165 of
 *                      the 343 cells of a 5^3 box), the halo cells staying
 *                      as they are.
 *   patch_offsets, patch_sizes  HOST arrays; offsets must ascend without
 *                      overlap (FV_ERR_INVALID_ARG), 16-byte multiples
 *                      (FV_ERR_ALIGNMENT); sizes in 1..max_patch_size
 *                      (FV_ERR_BAD_PATCH).
 *   dx, dt             as for fv_patch_update_batch (dt <= 0: the device
 *                      time step slot).
 * Synchronous: returns when host_out holds the whole result.  Starts after
 * the work already enqueued on the handle's stream.
 */
fv_status fv_patch_update_host(fv_batch* h, const void* host_in, void* host_out,
                               const int64_t* patch_offsets, const int32_t* patch_sizes,
                               int64_t n_patches, double dx, double dt, int64_t chunk_patches);

/*
 * fv_patch_update_local -- fv_patch_update_batch with a cell size and a time
 * step per patch (the batch descriptor of Sec. 3 carries both per patch):
 * patch i advances with Q - (dt_i / dx_i) sum (F_+ - F_-) (Eq. 3).
 *   dx_patch      device double[n_patches]: cell size of each patch (> 0).
 *   dt_patch      device double[n_patches]: with cfl <= 0 the time step of
 *                 each patch (input); with cfl > 0 each patch takes its own
 *                 CFL step dt_i = cfl * dx_i / (d * lambda_i), lambda_i the
 *                 maximum of a over its faces (Eq. 5; the per-patch value of
 *                 fv_max_eigenvalue_reduce), written here (output).
 *   lambda_patch  nullable device double[n_patches]: lambda_i.
 * Halos as for fv_patch_update_batch.  With all dx_i = dx and dt_i = dt the
 * result is bitwise that of fv_patch_update_batch.  Both arrays 8-byte
 * aligned (FV_ERR_ALIGNMENT), non-null (FV_ERR_INVALID_ARG).
 */
fv_status fv_patch_update_local(fv_batch* h, const void* in_with_halo, void* out,
                               const int64_t* patch_offsets, const int32_t* patch_sizes,
                               int64_t n_patches, const double* dx_patch, double* dt_patch,
                               double cfl, double* lambda_patch);

/*
 * Halos on a 3:1 refined mesh (the spacetree of Sec. 2 splits a cube into
 * three parts per axis; each cube carries a patch of p^d cells).  Patch i
 * sits on tree cell coord[i*d .. i*d+d-1] (x first, each in [0, 3^level))
 * of level level[i] (0..11) of the unit domain; all patches have size p.
 * A face-halo cell receives the mean of the neighbouring solution over its
 * region: the neighbour's cell (same level), the coarser neighbour's cell
 * that contains it (constant prolongation), or the mean of the 3^d finer
 * cells it covers (restriction); beyond a non-periodic domain edge the
 * rules of fv_halo_fill (boundary 0: periodic, -1 outflow, -2 wall).
 * Neighbouring tree cells may differ by one level (FV_ERR_INVALID_ARG
 * otherwise); meshes with more than one level need p >= 3
 * (FV_ERR_UNSUPPORTED).
 * fv_amr_plan_create -- builds the plan on the host (level, coord,
 *   patch_offsets: HOST arrays; offsets as for the other calls, 16-byte
 *   multiples) and copies it to the device; synchronous.
 * fv_amr_halo_fill -- fills the face halos of q_with_halo (device, the
 *   layout of the plan's offsets) on the handle's stream; interior cells are
 *   read, halo cells written.
 * fv_amr_plan_destroy -- frees the plan.
 */
typedef struct fv_amr_plan fv_amr_plan; /* opaque */
fv_status fv_amr_plan_create(fv_batch* h, fv_amr_plan** plan, int64_t n_patches,
                             const int32_t* level, const int32_t* coord,
                             const int64_t* patch_offsets, int p, int boundary);
fv_status fv_amr_halo_fill(fv_batch* h, const fv_amr_plan* plan, void* q_with_halo);
fv_status fv_amr_plan_destroy(fv_amr_plan* plan);

/*
 * fv_time_step -- one full explicit time step of a patch mesh in one kernel
 * launch: the update of fv_patch_update_batch (Eq. 3-5) with
 *   - dt = cfl * dx / (d * lambda) from the CFL condition on the current
 *     state's maximum wave speed lambda, which the handle holds on the
 *     device (left there by the previous fv_time_step, or by
 *     fv_max_eigenvalue_reduce on the initial state after its halo fill);
 *   - the face-halo cells read straight from the neighbours' interiors of
 *     in_with_halo by the rules of fv_halo_fill (neighbours as there), so
 *     the halo cells of both buffers are neither read nor written;
 *   - the maximum wave speed of Q^{n+1} (all interior cells, all directions)
 *     reduced on the device for the next step.
 * For a mesh closed by neighbours, outflow and walls this equals, bitwise,
 * fv_halo_fill + fv_max_eigenvalue_reduce + fv_patch_update_batch with
 * dt <= 0.  dt is also written to the handle's time step slot.
 * lambda_patch (nullable): per-patch max a over the faces used.
 */
fv_status fv_time_step(fv_batch* h, const void* in_with_halo, void* out,
                       const int64_t* patch_offsets, const int32_t* patch_sizes,
                       const int32_t* neighbours, int64_t n_patches, double dx, double cfl,
                       double* lambda_patch);

/*
 * Primitive carry between time steps.  A time step converts its new state
 * to primitives (u_1..u_d, p, c, E + p of every interior cell; Eq. 2) for
 * the next step's CFL condition anyway; handing them to the next step saves
 * that step the conversion of every interior and face-halo cell (about a
 * quarter of the FP64 work of a 3D step).
 *
 * fv_prim_stride -- elements (of the handle's precision) per patch of a
 * primitive buffer: (d + 3) * max_patch_size^d rounded up to 16 bytes.  A
 * buffer for n patches holds n * stride elements; patch i's block starts at
 * element i * stride: component m (u_1..u_d, p, c, E + p) of interior cell
 * (x, y, z) (0-based, x fastest) at m * p^d + x + p (y + p z).
 *
 * fv_time_step_prim -- fv_time_step with the carry: prim_in (device,
 * nullable) holds the primitives of in_with_halo as the previous
 * fv_time_step_prim wrote them to its prim_out; NULL computes them from the
 * state (the first step).  prim_out (device, nullable) receives the
 * primitives of out.  Both 16-byte aligned, n_patches * fv_prim_stride
 * elements, distinct (prim_in == prim_out is FV_ERR_INVALID_ARG).  The
 * caller owns them and must not change the state between the step that
 * wrote prim_out and the step that reads it as prim_in: stale primitives
 * give wrong fluxes (no error is detected).  The result is bitwise that of
 * fv_time_step.
 */
fv_status fv_prim_stride(const fv_batch* h, int64_t* elems_per_patch);
fv_status fv_time_step_prim(fv_batch* h, const void* in_with_halo, void* out,
                            const void* prim_in, void* prim_out, const int64_t* patch_offsets,
                            const int32_t* patch_sizes, const int32_t* neighbours,
                            int64_t n_patches, double dx, double cfl, double* lambda_patch);

/*
 * fv_run_steps -- n_steps time steps from q0: fv_halo_fill and
 * fv_max_eigenvalue_reduce on q0, then fv_time_step_prim ping-ponging
 * between q0 and q1.  FP64 handles carry the primitives from step to step in
 * two buffers the handle allocates on first use (2 * n_patches *
 * fv_prim_stride elements, kept until fv_batch_destroy; growing them drops
 * the cached graphs); FP32 handles run without the carry (faster there).
 * The result is in q0 if n_steps is even, else in q1.
 * use_graph != 0 captures the whole sequence into a CUDA graph the first
 * time a given set of arguments is seen, caches the instantiated graph in
 * the handle (keyed by every pointer and value argument) and replays it;
 * it needs a handle created on a non-default stream.  Buffers must not be
 * freed and reallocated at the same addresses while cached graphs refer to
 * them (fv_batch_destroy drops the cache).
 */
fv_status fv_run_steps(fv_batch* h, void* q0, void* q1, const int64_t* patch_offsets,
                       const int32_t* patch_sizes, const int32_t* neighbours, int64_t n_patches,
                       double dx, double cfl, int n_steps, int use_graph);

/*
 * Scheduling of batches with uneven patch sizes (the batched kernel of
 * Sec. 3 takes N patches of any sizes in one invocation).
 *   FV_SCHED_STRIDE   one persistent launch; CTA b takes patches b, b+G, ...
 *                     in index order; shared memory sized for the largest p.
 *                     The default, and the only one without a plan.
 *   FV_SCHED_LPT      one persistent launch over the patches sorted by size,
 *                     largest first (longest-processing-time-first order).
 *   FV_SCHED_CLASSES  one launch per patch size, each with the shared memory,
 *                     pipeline depth and occupancy of its own size.
 *   FV_SCHED_QUEUE    one persistent launch whose CTAs pop the patches, sorted
 *                     by size, largest first, from a work queue (a device
 *                     counter in the handle's workspace, zeroed by a kernel
 *                     enqueued before the launch): a CTA that finishes early
 *                     takes the next patch.
 * All four give bitwise identical results.  fv_batch_autotune chooses among
 * the first three.
 */
typedef enum {
  FV_SCHED_STRIDE = 0,
  FV_SCHED_LPT = 1,
  FV_SCHED_CLASSES = 2,
  FV_SCHED_QUEUE = 3
} fv_schedule;

/*
 * fv_batch_plan -- sorts the patches of a batch by size (a stable counting
 * sort: within a size the patches keep their index order; patch_sizes:
 * device int32[n_patches], read back to the host once) for the LPT and
 * CLASSES schedules, and keeps the plan in the handle.  Synchronises the
 * handle's stream (call it outside stream capture).  A later update or time
 * step uses the plan when it is given the same patch_sizes pointer and
 * n_patches; the caller re-plans if the sizes change.
 */
fv_status fv_batch_plan(fv_batch* h, const int32_t* patch_sizes, int64_t n_patches);

/*
 * fv_batch_set_wait_limit -- how many clock cycles a CTA of the step kernel
 * (the general update / time-step kernel; not the FP32 one-size kernels)
 * waits for the bulk copy of a patch before it gives up, sets the timeout bit
 * of the status word (fv_get_status then returns FV_ERR_TIMEOUT) and leaves
 * its remaining patches unwritten.  Every wait of the device code is bounded
 * this way; the default, about one second at 2 GHz (2e9 cycles), only runs
 * out if a copy never completes.  cycles <= 0 restores the default; larger
 * values are refused (FV_ERR_INVALID_ARG).  A smaller limit makes the timeout
 * path testable on healthy hardware: the waits for copies already in flight
 * after a wait gave up keep the full default limit, so no CTA exits with a
 * copy pending and the context stays usable.  Applies to launches made after
 * the call (a graph cached by fv_run_steps keeps the limit it was captured
 * with).  Not in the paper: the failure handling of the library.
 */
fv_status fv_batch_set_wait_limit(fv_batch* h, long long cycles);

/* Selects the schedule of later updates and time steps. */
fv_status fv_batch_set_schedule(fv_batch* h, fv_schedule schedule);

/*
 * Patch-to-thread mapping of the FV_SCHED_CLASSES launches: one CTA advances
 * one patch at a time with `threads` threads (32: a warp per patch, 64, 128
 * or 256: a CTA per patch), set per patch size p (1..max_patch_size).  The
 * default (also of launches without a plan) follows the patch size: 32
 * threads for up to 64 interior cells, 256 for 3D patches above 200 cells,
 * else 128; d = 1 supports 128 only (FV_ERR_UNSUPPORTED otherwise).
 * The mapping never changes the results (bitwise).  fv_batch_class_threads
 * reads the current choice.
 */
fv_status fv_batch_set_class_threads(fv_batch* h, int p, int threads);
fv_status fv_batch_class_threads(const fv_batch* h, int p, int* threads);

/*
 * FP32 handles with d = 3 or d = 2 run the launches whose patches all have
 * one of the sizes below (a size class of FV_SCHED_CLASSES, or a planned
 * batch of that one size under any schedule) on a kernel built for that
 * size: 3D p = 3 .. 7 (eight lanes a patch, a lane per row of cells, the
 * patch swept plane by plane along z) and 2D p = 3 .. 6 (eight lanes a
 * patch, a lane per row of cells).  They perform the same operations in the same order as the
 * general kernel, so results are bitwise identical; class thread settings do
 * not apply to them.  Not used with the primitive carry, flux corrections or
 * per-patch cell sizes.  fv_batch_pairs_launches returns how many launches
 * of the handle used one of them (host counter, no synchronisation).
 */
fv_status fv_batch_pairs_launches(const fv_batch* h, int64_t* launches);

/*
 * fv_batch_autotune -- first picks, for every size class of the batch, the
 * fastest of the CTA sizes 32, 64, 128 and 256 (one-class launches), then
 * times the three schedules on the caller's batch (one warm-up and three
 * timed fv_time_step calls each, or fv_patch_update_batch calls with
 * dt = cfl * dx when neighbours is NULL), keeps the fastest in the handle and
 * returns it in *chosen (nullable); ms_per_schedule (host double[3],
 * nullable) receives the average milliseconds of each.
 * Plans the batch first if needed.  scratch_out is overwritten; the
 * handle's wave speed and time step are restored afterwards.  Synchronises.
 */
fv_status fv_batch_autotune(fv_batch* h, const void* in_with_halo, void* scratch_out,
                            const int64_t* patch_offsets, const int32_t* patch_sizes,
                            const int32_t* neighbours, int64_t n_patches, double dx, double cfl,
                            fv_schedule* chosen, double* ms_per_schedule);

/*
 * Learned face-flux correction (the build's addition on top of Eq. 4; not in
 * the paper).  A network of 16 -> 64 -> 64 -> 4 units with GELU activations
 * maps the normalised 4-cell stencil Q_{i-2..i+1} normal to a face (in the
 * face's normal frame: rho, j_n, j_t, E per cell) to a correction C that is
 * added to the Rusanov flux of that face, once per face, so both cells see
 * the same flux and the totals are conserved by construction.
 * Parameters: one FP32 device vector of FV_MLP_NPARAM floats, in the order
 * W1 (64x16, output-major), b1 (64), W2 (64x64), b2 (64), W3 (4x64), b3 (4).
 * Normalisation: FP32 device vector of FV_MLP_NNORM floats: mu_x (16),
 * sd_x (16), sd_y (4); x = (stencil - mu_x) / sd_x, C = y * sd_y.
 * All products run on the tensor cores in BF16 with FP32 accumulation.
 */
#define FV_MLP_NPARAM 5508
#define FV_MLP_NNORM 36

typedef struct fv_mlp_trainer fv_mlp_trainer; /* opaque */

/*
 * The trainer: batches of up to max_batch samples, on cuda_stream (on the
 * current device).  The network kernel walks tiles of 128 samples, two CTAs
 * per SM, each CTA running forward, loss gradient, backward and the weight
 * gradients of its tiles on the tensor cores (tcgen05) and leaving one
 * partial gradient; a second kernel sums the partials in a fixed order and
 * applies Adam, so results are deterministic.  The trainer owns the partial
 * gradients (2 x SMs x FV_MLP_NPARAM floats), the Adam moments (zero at
 * creation) and a status word.  x and target (below) must be 16-byte
 * aligned (FV_ERR_ALIGNMENT otherwise).
 */
fv_status fv_mlp_trainer_create(fv_mlp_trainer** t, int64_t max_batch, void* cuda_stream);
fv_status fv_mlp_trainer_destroy(fv_mlp_trainer* t);

/* Synchronises the trainer's stream, reads and clears its status word:
 * FV_ERR_TIMEOUT if a kernel gave up waiting for its products (bounded
 * waits, about one second), else FV_OK. */
fv_status fv_mlp_trainer_status(fv_mlp_trainer* t);

/* y (device float[batch*4]) = network(x) for normalised inputs x
 * (device float[batch*16]). */
fv_status fv_mlp_forward(fv_mlp_trainer* t, const float* params, const float* x, int64_t batch,
                         float* y);

/* Mean squared error of network(x) against target (device float[batch*4])
 * into *loss (device float) and its gradient into grad (device
 * float[FV_MLP_NPARAM]); deterministic. */
fv_status fv_mlp_grad(fv_mlp_trainer* t, const float* params, const float* x,
                      const float* target, int64_t batch, float* grad, float* loss);

/* One Adam step (lr, step >= 1 counts the steps; moments kept in the
 * trainer) on params in place; *loss receives the batch loss before it. */
fv_status fv_mlp_train_step(fv_mlp_trainer* t, float* params, const float* x, const float* target,
                            int64_t batch, float lr, int step, float* loss);

/*
 * n_steps Adam steps (steps first_step .. first_step + n_steps - 1, each
 * counted as in fv_mlp_train_step) on consecutive minibatches of a sample set
 * already on the device: step k uses the batch rows starting at
 * ((k - 1) mod (n_samples / batch)) * batch of x (float[n_samples*16]) and
 * target (float[n_samples*4]).  losses (device float[n_steps], nullable)
 * receives each step's batch loss.  Two kernel launches per step, enqueued
 * without synchronisation.
 */
fv_status fv_mlp_train_steps(fv_mlp_trainer* t, float* params, const float* x,
                             const float* target, int64_t n_samples, int64_t batch,
                             int first_step, int n_steps, float lr, float* losses);

/*
 * Learned correction on 2D patch meshes (handles with d == 2 and patches of
 * at most 16 cells per axis).  Per-face arrays hold, per patch, the faces of
 * each direction k (x then y), each unknown v, face j = tr + p b (b the
 * halo-1 coordinate of the face's left cell along k, tr the transverse
 * interior index from 0): element [patch * fv_corr_stride(h) +
 * (k * 4 + v) * (p + 1) * p + j].
 */
/* Floats per patch of the per-face arrays: 8 (pmax + 1) pmax. */
int64_t fv_corr_stride(const fv_batch* h);

/*
 * fv_flux_correction -- C for every face of every patch of the state q (the
 * stencil cells outside a patch come from the neighbours by the rules of
 * fv_halo_fill, two layers deep), into corr (device float, fv_corr_stride(h)
 * per patch).  params: device float[FV_MLP_NPARAM]; norm: device
 * float[FV_MLP_NNORM].  Runs on the tensor cores (BF16, FP32 accumulate).
 * Each face of the mesh is evaluated once: a face shared by two patches that
 * name each other as neighbours along its direction takes the stencil of the
 * upper patch's face b = 0, and its C is written into both patches' slots
 * (bitwise the same values); a face with no such neighbour (wall, outflow, a
 * table that is not symmetric) is evaluated by its own patch.  Every slot of
 * a valid patch of size p is written; slots of sizes below the handle's
 * maximum are not.  Patches: at most 2^31 - 1 (FV_ERR_UNSUPPORTED above).
 */
fv_status fv_flux_correction(fv_batch* h, const void* q, const int64_t* patch_offsets,
                             const int32_t* patch_sizes, const int32_t* neighbours,
                             int64_t n_patches, const float* params, const float* norm,
                             float* corr);

/* fv_time_step with the face fluxes F + C, C from fv_flux_correction on the
 * same state (conservative: one F + C per face). */
fv_status fv_time_step_corrected(fv_batch* h, const void* in_with_halo, void* out,
                                 const int64_t* patch_offsets, const int32_t* patch_sizes,
                                 const int32_t* neighbours, int64_t n_patches, double dx,
                                 double cfl, const float* corr);

/*
 * Training data of the correction, on regular periodic 2D meshes: patches of
 * one size per mesh, patch index a + px b (x fastest), the fine mesh covering
 * the same domain at `ratio` times the resolution; the fine handle is FP64.
 * fv_restrict_mesh        coarse interior cells = means of their ratio^2 fine
 *                         cells;
 * fv_accumulate_face_flux acc[face] += weight * mean of the ratio fine
 *                         Rusanov fluxes on each coarse face (acc: device
 *                         double, fv_corr_stride(hc) per coarse patch; the
 *                         fine halos must be filled);
 * fv_correction_samples   per coarse face (sample = patch * 2 (p+1) p +
 *                         k (p+1) p + j): the raw 16-value stencil x_raw and
 *                         the target C* = acc - F_Rusanov(coarse state) t_raw
 *                         (4 values), both in the face's normal frame; FP64
 *                         coarse handle.
 */
fv_status fv_restrict_mesh(fv_batch* h_fine, const void* q_fine, const int64_t* off_fine,
                           int px_fine, int py_fine, fv_batch* h_coarse, void* q_coarse,
                           const int64_t* off_coarse, int px_coarse, int py_coarse, int ratio);
fv_status fv_accumulate_face_flux(fv_batch* h_fine, const void* q_fine, const int64_t* off_fine,
                                  int px_fine, int py_fine, fv_batch* h_coarse, int px_coarse,
                                  int py_coarse, int ratio, double weight, double* acc);
fv_status fv_correction_samples(fv_batch* h_coarse, const void* q_coarse,
                                const int64_t* patch_offsets, const int32_t* patch_sizes,
                                const int32_t* neighbours, int64_t n_patches, const double* acc,
                                float* x_raw, float* t_raw);
/* Column sums and sums of squares (FP64) of a row-major float matrix;
 * scratch: device double[2 cols ceil(rows / 65536)]. */
fv_status fv_column_moments(const float* x, int64_t rows, int cols, double* sum, double* sumsq,
                            double* scratch, void* cuda_stream);
/* x[r][c] = (x[r][c] - mu[c]) / sd[c] in place (mu nullable: 0). */
fv_status fv_normalize_columns(float* x, int64_t rows, int cols, const float* mu, const float* sd,
                               void* cuda_stream);

/*
 * fv_conserved_totals -- FP64 sums over all interior cells of every unknown
 * (mass, momentum, energy), for conservation checks.  Fixed-order two-stage
 * reduction (per patch, then per block, then one block), so the result is
 * bitwise reproducible.  FP32 handles accumulate in FP64.
 *   totals  device double[s].
 */
fv_status fv_conserved_totals(fv_batch* h, const void* q_with_halo, const int64_t* patch_offsets,
                              const int32_t* patch_sizes, int64_t n_patches, double* totals);

/*
 * fv_patch_sums -- the per-patch stage of fv_conserved_totals written out:
 * the FP64 sum of every unknown over each patch's interior cells (the
 * conservation epilogue of Algorithm 1's update, per patch), in the same
 * fixed order, so the totals are the fixed-order sum of these.
 *   per_patch  device double[n_patches][s], 8-byte aligned
 *              (FV_ERR_ALIGNMENT); row i holds patch i's sums; rows of
 *              invalid patches (bad size or offset: the status word's
 *              bad-patch bit) are left as they are.
 *   totals     device double[s] or NULL: as fv_conserved_totals.
 */
fv_status fv_patch_sums(fv_batch* h, const void* q_with_halo, const int64_t* patch_offsets,
                        const int32_t* patch_sizes, int64_t n_patches, double* per_patch,
                        double* totals);

/*
 * fv_conserved_totals_noalloc -- the sums of fv_conserved_totals for callers
 * that cannot allocate device memory (no counterpart in the paper).  Some
 * callers own the whole GPU through their own memory pool and forbid any
 * other allocation, or run latency-critical loops in which cudaMalloc or
 * cudaFree would synchronise the device; they cannot create an fv_batch,
 * whose workspace is allocated.  This entry point needs no handle and
 * allocates nothing: it calls no cudaMalloc, cudaFree or allocating library
 * routine.  Its scratch (the per-chunk partial sums) is a static device
 * array of 256 KiB inside libfv.so, held on every device that loads the
 * library until the process exits.
 *   d, s, precision  as for fv_batch_create (s == d + 2); halo width 1;
 *                    patch sizes in [1, 64].
 *   q_with_halo, patch_offsets, patch_sizes, n_patches  as for
 *                    fv_conserved_totals; n_patches <= 4,194,304
 *                    (4096 chunks of 1024 patches); larger batches return
 *                    FV_ERR_UNSUPPORTED and enqueue nothing.
 *   totals           device double[s], written.
 *   status_word      device unsigned int, required (NULL returns
 *                    FV_ERR_INVALID_ARG: the library keeps no status word
 *                    that such a caller could read); bad-patch (1) and
 *                    non-physical (2) bits are OR-ed into it, never cleared.
 *   cuda_stream      cudaStream_t to enqueue on (NULL: legacy default stream).
 * The first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress) and caches it; make that first call
 * before any stream capture.  Every call on a device shares the one array;
 * each call writes every partial slot it reads before reading it, so no
 * slot needs clearing, but calls that overlap on the GPU (two streams, two
 * threads) race on the array and give wrong totals: serialise them.
 * Results are bitwise equal to fv_conserved_totals on the same input.
 */
fv_status fv_conserved_totals_noalloc(int d, int s, fv_precision precision,
                                      const void* q_with_halo, const int64_t* patch_offsets,
                                      const int32_t* patch_sizes, int64_t n_patches,
                                      double* totals, unsigned int* status_word,
                                      void* cuda_stream);

/* Device address of the handle's time step slot (double[1]). */
fv_status fv_get_dt_ptr(fv_batch* h, double** dt_device);

/* Synchronises the handle's stream and copies its time step slot (the dt of
 * the last reduce or time step) to *dt_host. */
fv_status fv_read_dt(fv_batch* h, double* dt_host);

/*
 * fv_get_status -- synchronises the handle's stream, reads and clears the
 * device status word and returns the first error it records (FV_ERR_BAD_PATCH,
 * FV_ERR_NONPHYSICAL, FV_ERR_TIMEOUT), or the first CUDA error, else FV_OK.
 */
fv_status fv_get_status(fv_batch* h);

/* Text of the last error on this handle ("" if none).  Owned by the handle. */
const char* fv_last_error(const fv_batch* h);

/* Static text naming a status code. */
const char* fv_status_string(fv_status s);

/*
 * Diagnostics (no counterpart in the paper).
 * fv_selftest_math -- evaluates, on the current device and the legacy
 * default stream, the FP64 reciprocal (which == 0) or square root
 * (which == 1) that the FP64 kernels use for 1/rho and the sound speed, on
 * n device doubles x, into the device doubles out; synchronises.  Lets
 * tests measure their error against the IEEE operations.
 */
fv_status fv_selftest_math(const double* x, double* out, int64_t n, int which);

#ifdef __cplusplus
}
#endif
#endif /* FV_H */
