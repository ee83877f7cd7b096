/*
 * raytrax.h -- C ABI of the GB300 (sm_103a) emission-absorption ray march.
 *
 * The library implements the single-source kernel and its multi-source / multi-bin wrapper
 * of the paper (Sec. 2, "Method and code structure" and "Frequency-bin agnosticism"):
 * from every source, N_Omega rays on a Fibonacci (golden-angle) lattice march N_s substeps
 * of Eq. 2,
 *       x_{k+1} = x_k + n ds,  tau_{k+1} = tau_k + kappa(x_k) ds,
 *       I_{k+1} = I_k exp(-kappa(x_k) ds) + j(x_k) exp(-tau_k) ds,
 * with j read trilinearly at x_k, kappa read at the nearest cell of x_k, and I_{k+1}
 * deposited back with the same trilinear weights, indices clamped to the box. Deposits are
 * scaled by 4 pi / N_Omega and summed over rays, sources and substeps, per frequency bin.
 *
 * Conventions shared by every entry point:
 *   - Grids are float32, C-contiguous, shape [n_freq][n0][n1][n2]; bins are independent.
 *   - Grid coordinates are node-centred: voxel (i0, i1, i2) sits at point (i0, i1, i2).
 *     Component a of a position or direction indexes array axis a.
 *   - Per axis, f = floor(x), corners clamp(f, 0, n-1) and clamp(f+1, 0, n-1), fraction
 *     t = x - f (unclamped); a ray that leaves the box keeps marching and deposits on the
 *     nearest boundary voxels.
 *   - kappa cell: kappa_mode 0 = the clamped floor corner of x_k (default); kappa_mode 1 =
 *     clamped floor(x_k + 1/2). The paper fixes only a nearest-neighbour read at the cell of
 *     the previous position, not which cell that is.
 *   - Lattice: z_i = 1 - (2i+1)/N, phi_i = i pi (3 - sqrt 5) mod 2 pi, n_i = (sqrt(1-z^2)
 *     cos phi, sqrt(1-z^2) sin phi, z), computed in FP64 and rounded once to FP32.
 *   - Geometry in IEEE FP32 without contraction: d = fl(n ds) once per ray,
 *     x_{k+1} = fl(x_k + d), t = fl(x - floor x); so cell indices are reproducible.
 *   - N_s = ceil(c dt / ds) evaluated in FP64 from the float arguments (relative guard
 *     1e-9 against roundoff), then min(N_s, ns_cap) when ns_cap > 0.
 *   - "device" pointers are CUDA global-memory pointers of the current device; every
 *     device call is asynchronous on the given stream (NULL = legacy default stream).
 *     The caller owns every data buffer; a handle owns only its scratch (direction
 *     tables, packed inputs, accumulators, checkpoints), freed by rt_destroy.
 *   - Errors found on the host return at once with nothing enqueued; the thread-local
 *     message of rt_last_error() says which argument. CUDA launch or allocation failures
 *     return RT_ERR_CUDA / RT_ERR_OOM. A handle may be used by one host thread at a time.
 */
#ifndef RAYTRAX_H
#define RAYTRAX_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rt_grid rt_grid;

typedef enum {
    RT_OK = 0,
    RT_ERR_INVALID_ARG = 1,
    RT_ERR_CUDA = 2,
    RT_ERR_OOM = 3,
    RT_ERR_TIMEOUT = 4,
    RT_ERR_INTERNAL = 5,
    RT_ERR_UNSUPPORTED = 6
} rt_status;

typedef struct {
    int deterministic;  /* 0: FP32 atomic accumulation (default). 1: every deposit is rounded
                           to a 64-bit fixed-point integer (unit 1 / 2^k with the largest k that
                           keeps the a-priori bound 4 pi N_src ds max|j| N_s (N_s+1) / 2 below
                           2^62; needs kappa >= 0) and added as an integer: rt_advance's field is
                           bitwise identical for every launch plan and deposit order.
                           rt_advance / rt_advance_rays only (no autotuning, no batch). Honours
                           plan_width and plan_block; rt_create_grid rejects plan_lanes 2,
                           plan_tile 2 and plan_prefetch other than 0, 1 or 5 with it (one lane
                           per ray, corner slots -- gathers mode 0 or 4, which sum alike -- and no
                           tiles). */
    int kappa_mode;     /* 0: floor cell of x_k (default); 1: round-to-nearest cell */
    int ns_cap;         /* 0: none; > 0: cap on the substep count (the optional cap of Sec. 2) */
    int autotune;       /* 1: time the launch shapes once per shape class and keep the best */
    int ckpt_stride;    /* adjoint checkpoint stride K in substeps, rounded to 4, 8, 16 or 32;
                           0: automatic -- with autotune = 1 the first rt_backward* of each shape
                           class (n_freq, sources, rays, N_s) times the reverse march for every K
                           on its own inputs (synchronising the stream) and keeps the fastest for
                           that class, its recordings included; otherwise 16 */
    int profile;        /* 1: bracket the march kernel of each call with CUDA events on the
                           call's stream, readable with rt_kernel_ms */
    /* Forward launch plan, used when autotune = 0; 0 in a field means that field's default.
       plan_width: bins per group (1, 2 or 4). plan_block: threads per block (32..256, a
       multiple of 32). plan_prefetch: gathers mode + 1, where mode 0 keeps the 8 corners in
       slots (when the ray crosses a face, the 4 corners on it keep their gathered j and their
       summed deposits; the other 4 are flushed and re-gathered), mode 1 issues the next
       substep's gathers before the current update, mode 2 does both, mode 3 reuses the
       whole corner set while it is unchanged and flushes and re-gathers all 8 corners when it
       changes, and mode 4 is mode 0 with the corners that enter at substep k+1 gathered before
       the update of substep k (no tiles). plan_lanes: lanes per ray (1, or 2 adjacent lanes
       sharing one ray, each keeping the four corner slots on its side of axis 2, for twice the
       warps; gathers mode 0 or 4). plan_tile: source deposit tiles (1: off, 2: on): each
       block sums the deposits of its rays in the 8^3 cells around its source in shared memory
       and adds them to the field once (FP32 sums only; not in deterministic mode). */
    int plan_width;
    int plan_block;
    int plan_prefetch;
    int plan_lanes;
    int plan_tile;
    int check_inputs;   /* 1: checked mode. rt_advance* and rt_backward* first scan j, kappa,
                           the sources (and grad_out) on the device and return
                           RT_ERR_INVALID_ARG, naming the array, if a value is not finite, a
                           kappa is negative or a source coordinate has |x| >= 2^24. The scan
                           synchronises the stream (one pass over the inputs). 0: no scan. */
    int record_checkpoints; /* 1: every full-range rt_advance also stores the reverse march's
                           checkpoints (every ckpt_stride substeps) in the handle, marching
                           with the adjoint's bin grouping (one bin: two lanes per ray; wider
                           groups: one lane; both with gathers mode 4) unless a plan is pinned
                           (with autotune = 1: the fastest plan that records, timed with its
                           checkpoint stores, tuned apart from non-recording calls); a following
                           rt_backward / rt_backward_sources with the same j_map, kappa_map and
                           source_pos pointers and the same scalars uses them instead of
                           repeating the forward sweep -- but only if a 64-bit content hash of
                           j, kappa and the sources, taken on the device at the forward and again
                           at the backward, is unchanged (decided on the device, no
                           synchronisation): buffers rewritten in place in between get the
                           gradients of their new contents. 0: off. */
    int accumulation;   /* how deposits are summed into the field (deterministic = 1 implies 3):
                           0: automatic (default): FP32 while the call deposits fewer than 32
                              updates per cell and bin on average (num_sources * num_rays * N_s
                              < 32 * n0 n1 n2); denser calls, where FP32 sums lose the small
                              deposits to rounding, sum in 64-bit fixed point -- or in FP64 where
                              the fixed-point unit would be coarse (num_sources * N_s (N_s + 1) / 2
                              above 2^32) and in rt_advance_continue.
                           1: FP32 reductions (W-wide vectors). A cell that takes very many
                              small deposits on top of a large sum -- next to many clustered
                              sources, on the clamped box corners -- loses them to rounding:
                              relative L2 error ~1e-4 on 2,097 clustered sources.
                           2: FP64 reductions (one per bin), converted to FP32 once.
                           3: 64-bit fixed point as in deterministic mode (unit: the bound given
                              there over 2^62; needs kappa >= 0), any launch plan that has it.
                           Sums in 8-byte words take no source tiles (a plan that pins them keeps
                           FP32 in the automatic mode). Fixed-point sums are independent of the
                           deposit order, FP64 ones up to FP64 rounding. rt_advance_noalloc and
                           batches sum in FP32. */
} rt_options;

/* Fill *opt with the defaults (all zero: FP32 atomics, floor kappa cell, no cap,
   no autotuning, automatic checkpoint stride). */
void rt_default_options(rt_options* opt);

/* Create a handle for grids of n0 x n1 x n2 voxels and up to max_freq bins.
   n0, n1, n2 >= 1, max_freq >= 1, n_freq * n0 * n1 * n2 < 2^31; opt may be NULL (defaults).
   Allocates nothing on the device until the first call that needs scratch.
   *out receives the handle (NULL on error). */
rt_status rt_create_grid(rt_grid** out, int n0, int n1, int n2, int max_freq, const rt_options* opt);

/* Free the handle and its scratch after synchronising the device. NULL is accepted. */
rt_status rt_destroy(rt_grid* grid);

/* Thread-local description of the last error returned on this thread ("" if none). */
const char* rt_last_error(void);

/* N_s for (step_size, radiation_velocity, time_step) and a cap (<= 0: none), computed as
   described above; -1 if step_size <= 0, radiation_velocity <= 0, time_step < 0, a value
   is not finite or N_s would not fit in an int. Paper: Sec. 2 after Eq. 2; App. A. */
int rt_num_substeps(float step_size, float radiation_velocity, float time_step, int ns_cap);

/* Write the FP32 Fibonacci lattice (Sec. 2) used by the march, in lattice order, to the
   HOST buffer out[num_rays][3]. num_rays >= 1. */
rt_status rt_direction_table(int num_rays, float* out);

/* One time step dt of the field (Sec. 2: the single-source kernel's arguments
   (j_map, kappa_map, source_pos, num_rays, step_size, radiation_velocity, time_step),
   looped over sources and batched over n_freq bins):
     out_field[b] (+)= (4 pi / num_rays) sum_sources sum_rays sum_{k < N_s} W(x_k) I_{k+1}.
   j_map, kappa_map, out_field: device [n_freq][n0][n1][n2] float32 (kappa >= 0 expected).
   source_pos: device [num_sources][3] float32, grid coordinates, each |x| < 2^24.
   num_sources >= 0 (0 gives a zero field), num_rays >= 1, step_size > 0,
   radiation_velocity > 0, time_step >= 0, 1 <= n_freq <= max_freq.
   accumulate = 0 overwrites out_field, 1 adds to it. out_field must not alias j_map or
   kappa_map. Stream-ordered; the inputs must stay valid until the work completes. */
rt_status rt_advance(rt_grid* grid, const float* j_map, const float* kappa_map,
                     const float* source_pos, int num_sources, int num_rays,
                     float step_size, float radiation_velocity, float time_step, int n_freq,
                     float* out_field, int accumulate, void* cuda_stream);

/* rt_advance restricted to the lattice directions ray_begin .. ray_end-1 (each still
   weighted 4 pi / num_rays): the direction shard of Sec. 2 (each device marches a subset
   of the directions; the partial fields are summed). Shards that tile
   [0, num_rays) sum to the rt_advance field. 0 <= ray_begin <= ray_end <= num_rays. */
rt_status rt_advance_rays(rt_grid* grid, const float* j_map, const float* kappa_map,
                          const float* source_pos, int num_sources, int num_rays,
                          int ray_begin, int ray_end, float step_size, float radiation_velocity,
                          float time_step, int n_freq, float* out_field, int accumulate,
                          void* cuda_stream);

/* Stateful advance: the march continued across calls, for time integration with a fixed dt
   (Sec. 3: a fixed dt, advanced call after call; the light-travel horizon of Sec. 2 then grows
   by c dt per call). Same arguments and field as rt_advance, except that each ray starts where this
   handle's previous rt_advance_continue call left it -- at its position, with the intensity I
   and optical depth tau it had -- marches N_s = ceil(c dt / ds) further substeps through THIS
   call's j and kappa (which may change between calls), and deposits only those. The handle
   keeps the state: positions [num_sources][num_rays][3] and I, tau [n_freq][num_sources]
   [num_rays] in FP32 (20 bytes per lane and bin). The rays restart at their sources with
   I = tau = 0 when restart != 0, on the first call, and whenever num_sources, num_rays, n_freq
   or step_size differ from the previous call's (source positions must not change between
   continued calls). For the same j and kappa, n consecutive calls add up to one call over the
   summed substeps; the positions repeat the uninterrupted march's FP32 additions exactly.
   RT_ERR_UNSUPPORTED in deterministic mode. Not stream-safe across handles sharing state: one
   handle, one sequence of calls. */
rt_status rt_advance_continue(rt_grid* grid, const float* j_map, const float* kappa_map,
                              const float* source_pos, int num_sources, int num_rays, float step_size,
                              float radiation_velocity, float time_step, int n_freq, float* out_field,
                              int accumulate, int restart, void* cuda_stream);

/* rt_advance with HOST buffers (same shapes): copies the inputs to handle-owned device
   scratch, runs the march on the given stream, copies the field back and synchronises
   the stream before returning. Host buffers may be pageable; pinned ones copy faster. */
rt_status rt_advance_host(rt_grid* grid, const float* j_map, const float* kappa_map,
                          const float* source_pos, int num_sources, int num_rays,
                          float step_size, float radiation_velocity, float time_step, int n_freq,
                          float* out_field, void* cuda_stream);

/* Pipelined rt_advance_host: same arguments and field, but the call only ENQUEUES the work and
   returns. Three streams overlap consecutive calls: the inputs are copied in on a copy stream of
   the handle, the march runs on cuda_stream, the field is copied out on a second copy stream of
   the handle; two sets of device buffers alternate, so call i+1's inputs move in and call i-1's
   field moves out while call i marches. Calls complete in order. The host buffers must stay
   valid, and the inputs unmodified, until rt_host_wait returns (or until a stream joined with
   rt_host_join has passed the join); the field is in out_field only then. Consecutive calls may
   pass the same out_field (its copies land in call order). Pinned (page-locked) host buffers are
   needed for the copies to overlap anything; pageable ones work but serialise. The handle's
   other entry points share its march scratch: on the same cuda_stream they are ordered after
   the enqueued marches; on another stream, call rt_host_wait first. Errors of the enqueued work
   surface in rt_host_wait. */
rt_status rt_advance_host_async(rt_grid* grid, const float* j_map, const float* kappa_map,
                                const float* source_pos, int num_sources, int num_rays,
                                float step_size, float radiation_velocity, float time_step,
                                int n_freq, float* out_field, void* cuda_stream);

/* Block until every rt_advance_host_async call of this handle has finished, including its
   copy to the host; RT_ERR_CUDA if any of that work failed. */
rt_status rt_host_wait(rt_grid* grid);

/* Make cuda_stream (NULL: legacy default stream) wait, on the device, for every
   rt_advance_host_async call enqueued so far; the host does not block. */
rt_status rt_host_join(rt_grid* grid, void* cuda_stream);

/* Reverse-mode adjoint of rt_advance (the Jacobians w.r.t. (j, kappa) of Sec. 4,
   "Coupling to differentiable hydro"). Given grad_out = dL/d(out_field) (device,
   [n_freq][n0][n1][n2]) and the forward's inputs, writes dL/dj to grad_j and dL/dkappa
   to grad_kappa (device, same shape, OVERWRITTEN; either may be NULL to skip it).
   Per ray, with a_k = exp(-kappa_k ds), E_k = exp(-tau_k), s = 4 pi / num_rays:
     lam_{k+1} = s sum_c w_{k,c} G[c_{k,c}] + a_{k+1} lam_{k+2},
     mu_k = mu_{k+1} + lam_{k+1} j_k E_k ds,
     dj[c_{k,c}] += lam_{k+1} E_k ds w_{k,c},
     dkappa[cell_k] += -ds (lam_{k+1} I_k a_k + mu_{k+1}).
   The forward state is recomputed from per-ray checkpoints every ckpt_stride substeps
   (never by dividing out exp(-kappa ds)). For source positions see rt_backward_sources; not
   differentiable in ds, c, dt. */
rt_status rt_backward(rt_grid* grid, const float* grad_out, const float* j_map,
                      const float* kappa_map, const float* source_pos, int num_sources,
                      int num_rays, float step_size, float radiation_velocity, float time_step,
                      int n_freq, float* grad_j, float* grad_kappa, void* cuda_stream);

/* rt_backward plus the gradient with respect to the source positions: grad_src (device
   [num_sources][3], overwritten, or NULL). Sec. 4 notes that the march is built from smooth
   interpolation and deposition primitives; source positions enter only through them. Every
   position of a ray is x_k = src + k n ds, so dL/dsrc sums dL/dx_k over the source's rays
   and substeps with everything else fixed, where x_k enters the deposit of I_{k+1} and the
   gather of j:
     dL/dx_k = grad_x [ sum_c w_c(x) (s I_{k+1} G[c] + lam_{k+1} E_k ds j[c]) ] at x = x_k,
   the corner values held fixed. The nearest-cell kappa read is piecewise constant and adds
   nothing (the gradient is that of the almost-everywhere derivative); a clamped axis adds
   nothing. Any of grad_j, grad_kappa, grad_src may be NULL; they must not alias each other or
   an input. Summed with FP32 atomics (one per warp and component). */
rt_status rt_backward_sources(rt_grid* grid, const float* grad_out, const float* j_map,
                              const float* kappa_map, const float* source_pos, int num_sources,
                              int num_rays, float step_size, float radiation_velocity, float time_step,
                              int n_freq, float* grad_j, float* grad_kappa, float* grad_src,
                              void* cuda_stream);

/* Emissivity inversion (Sec. 4, gradient-based inversion, with every voxel of j free instead of
   one amplitude): starting from the j in j_map, `iterations` projected Adam steps (beta1 0.9,
   beta2 0.999, epsilon 1e-8, learning rate lr; after each step j = max(j, 0)) on
       L(j) = mean over the n_freq * n0 n1 n2 values of (log(F(j) + eps) - log(target + eps))^2,
       eps = eps_rel * max(target),
   where F(j) = rt_advance(j, kappa_map, source_pos, ...) with this call's scalars and dL/dj comes
   from rt_backward. target, kappa_map, j_map: device [n_freq][n0][n1][n2] (target >= 0, the
   field to match); j_map is overwritten with the recovered j. losses: device float
   [iterations + 1], overwritten: losses[i] = L before step i + 1, losses[iterations] = L of the
   result. Everything is enqueued on cuda_stream (NULL: legacy default stream) with no host
   synchronisation after the grid's first call of this shape class (autotuning, when on, times
   its plans then); a grid created with record_checkpoints = 1 lets each reverse march reuse the
   forward's checkpoints. Workspace: 6 n floats held by the grid. Errors: RT_ERR_INVALID_ARG for
   a NULL array, iterations < 0, lr or eps_rel not finite and positive, n_freq outside
   [1, max_freq], j_map aliasing an input or losses overlapping an array, and whatever
   rt_advance / rt_backward return for the problem's arguments. */
rt_status rt_invert_emissivity(rt_grid* grid, const float* target, const float* kappa_map,
                               const float* source_pos, int num_sources, int num_rays, float step_size,
                               float radiation_velocity, float time_step, int n_freq, int iterations,
                               float lr, float eps_rel, float* j_map, float* losses, void* cuda_stream);

/* Duration in ms of the march kernel(s) of the last rt_advance / rt_backward call on this
   handle (forward: the march kernel only, without packing or zeroing; backward: the adjoint
   kernel). Needs rt_options.profile = 1; waits for that kernel to finish. */
rt_status rt_kernel_ms(rt_grid* grid, float* ms);

/* Allocation-free forward march. The paper has no counterpart: this entry point exists for
   callers that cannot allocate memory while they run -- a program whose GPU memory belongs to
   another framework's pool or a fixed budget, or a loop that must never block in an allocator.
   It computes exactly what rt_advance computes (default options: kappa_mode 0, no N_s cap)
   for the same arguments, without a handle, and calls no cudaMalloc / cudaFree or any other
   allocating routine. Its scratch (sorted direction table, packed inputs, accumulator) is one
   static device array of RT_NOALLOC_SCRATCH_BYTES inside this library, which every GPU that
   loads the library holds until the process exits. Limits: num_rays <= RT_NOALLOC_MAX_RAYS,
   and for n_freq >= 2, 3 * ceil(n_freq / W) * W * n0 * n1 * n2 * 4 bytes (W = 2 for two bins,
   else 4) must fit in the rest of the array after the 256 KiB table (e.g. 64^3 with 4 bins);
   larger problems return RT_ERR_INVALID_ARG with the sizes in rt_last_error(). One bin needs
   only the table. Under CUDA's default lazy module loading, the array and the kernels' code
   are committed on a device by the first call there (with that device current), so that
   first call can still fail for lack of memory: callers that must allocate nothing later
   should make one warm-up call per device at start-up. Every call looks up the array's
   device address (and starts afresh if the device's context was replaced, e.g. after
   cudaDeviceReset); a call with a new num_rays, and the first call in a context, waits for the
   stream, rebuilds the table and copies it in stream order, then waits again: make such calls
   before any stream capture. All calls share the array
   and it keeps the last call's contents (the accumulator is cleared on the stream at every
   call); calls whose GPU work overlaps (other streams or host threads) race on it.
   Buffers, shapes and stream as in rt_advance; out_field is overwritten. */
#define RT_NOALLOC_SCRATCH_BYTES (16u << 20)
#define RT_NOALLOC_MAX_RAYS 16384
rt_status rt_advance_noalloc(const float* j_map, const float* kappa_map, const float* source_pos,
                             int num_sources, int n0, int n1, int n2, int num_rays, float step_size,
                             float radiation_velocity, float time_step, int n_freq, float* out_field,
                             void* cuda_stream);

/* ---- Batched persistent launch ----------------------------------------------------------
   Many independent march problems (each its own grid shape, sources, lattice size, bins and
   step) advanced by one persistent kernel, the whole run captured once in a CUDA graph. */
typedef struct rt_batch rt_batch;

typedef struct {
    const float* j_map;          /* device [n_freq][n0][n1][n2] */
    const float* kappa_map;      /* device, same shape */
    const float* source_pos;     /* device [num_sources][3], grid coordinates */
    int num_sources;             /* >= 1 */
    int n0, n1, n2, n_freq;      /* >= 1 each */
    int num_rays;                /* >= 1 */
    float step_size, radiation_velocity, time_step;   /* as in rt_advance */
    float* out_field;            /* device, same shape as j_map, OVERWRITTEN by each run */
} rt_instance;

/* Validate the instances, allocate the batch's scratch (packed copies, accumulators, lattice
   tables, work queue) and split the instances in two. An instance with at least
   RT_BATCH_DEDICATED_LANES (source, ray, bin group) lanes fills the GPU alone: it gets its own
   pack / march / unpack launches with a single-call launch plan. The others share persistent
   march kernels fed by work queues of 32-ray items (longest first), in waves whose packed
   inputs and accumulators fit in half the L2 cache. The buffers named in inst[] are bound to
   the batch: each rt_batch_run reads and writes them in place. opt: kappa_mode is honoured;
   autotune = 1 times, on the first run, the launch plans of the dedicated instances and the
   persistent block sizes. Same results as one rt_advance per instance. */
#define RT_BATCH_DEDICATED_LANES 19456
rt_status rt_batch_create(rt_batch** out, const rt_instance* inst, int n_inst, const rt_options* opt);

/* Advance every instance by its dt on the stream. The first call (optionally autotunes and)
   captures clear / pack / persistent march / unpack into a CUDA graph on an internal stream;
   every call then launches that graph on `cuda_stream` (NULL: legacy default stream). */
rt_status rt_batch_run(rt_batch* batch, void* cuda_stream);

/* One-shot batch: rt_batch_create with the handle's options (deterministic mode is not
   supported), one rt_batch_run on the stream, a synchronisation of the stream, and
   rt_batch_destroy. The instances need not match the handle's grid shape. For repeated runs
   keep an rt_batch: its CUDA graph is captured once. */
rt_status rt_advance_batch(rt_grid* grid, const rt_instance* inst, int n_inst, void* cuda_stream);

/* Total updates (substeps x rays x sources x bins over all instances) of one run. */
long long rt_batch_updates(const rt_batch* batch);

/* How instance `instance` (its index in rt_batch_create's array) is marched: *dedicated = 1
   for its own launches, then *width, *block, *prefetch, *tile give its plan (as rt_last_plan;
   final after the first rt_batch_run when autotuning); *dedicated = 0 for the persistent
   kernels, then *width = its bin-group width, *block = the persistent block size, *prefetch =
   *tile = 0. Any output may be NULL. RT_ERR_INVALID_ARG for a bad batch or index. */
rt_status rt_batch_info(const rt_batch* batch, int instance, int* dedicated, int* width, int* block,
                        int* prefetch, int* tile);

/* Free the batch (synchronises the device). NULL is accepted. */
rt_status rt_batch_destroy(rt_batch* batch);

/* ---- Convolutional surrogate: building blocks ----------------------------------------
   A 3-D CNN maps (log kappa, log(1 + j)) to the log of the field. Its 3x3x3 convolutions run on
   the tensor cores (tcgen05, BF16 operands, FP32 accumulate). Activations use the C32 layout:
   bf16 [B][D][H][W][32], 32 channels (64 bytes) per voxel, channels beyond the real count C
   zero, so every activation buffer holds B * D*H*W * 32 bf16 whatever C is (1 <= C <= 32).
   The convolution is the "same" cross-correlation with zero padding and dilation d:
     y[b][o][p] = bias[o] + sum_{i, tap} w[o][i][tap] x[b][i][p + (tap - centre) * d].
   All buffers are device memory; calls are asynchronous on the stream. */

/* FP32 [B][C][D][H][W] -> C32 (all 32 channels written), and back (the first C channels). */
rt_status rt_c32_from_f32(const float* src, int B, int C, int D, int H, int W, void* dst, void* cuda_stream);
rt_status rt_c32_to_f32(const void* src, int B, int C, int D, int H, int W, float* dst, void* cuda_stream);

/* Pack FP32 weights w[c_out][c_in][27] (tap = kz*9 + ky*3 + kx) into the kernel's bf16 layout
   [27][32][32] = [tap][n][k], 27 * 1024 bf16, unused entries zero. transpose = 0: for the forward
   convolution (n = output, k = input channel). transpose = 1: for the data gradient, the
   convolution with flipped taps that maps c_out channels back to c_in (n = input channel of the
   forward layer, k = its output channel). 1 <= c_in, c_out <= 32. */
rt_status rt_conv3d_pack_weights(const float* w, int c_in, int c_out, int transpose, void* packed,
                                 void* cuda_stream);

/* One convolution layer on the tensor cores. x: C32; w_packed from rt_conv3d_pack_weights;
   bias [c_out] or NULL; act 0 = identity, 1 = LeakyReLU(slope). mask (C32, or NULL): outputs
   where mask <= 0 are multiplied by slope before the activation (the LeakyReLU derivative when
   back-propagating). Outputs: y (C32, channels >= c_out written as 0) and/or y_f32
   ([B][D][H][W], FP32 channel 0). Requires W == 64, even H, 1 <= c_in, c_out <= 32; x must be
   16-byte aligned (a cudaMalloc pointer is). Waits inside the kernel are bounded: a timeout is
   reported by rt_device_status. */
rt_status rt_conv3d_forward(const void* x, int B, int D, int H, int W, int c_in, const void* w_packed,
                            const float* bias, int c_out, int dilation, int act, float slope,
                            const void* mask, void* y, float* y_f32, void* cuda_stream);

/* Weight and bias gradients of rt_conv3d_forward for dz = dL/d(pre-activation output):
     dw[co][ci][tap] += sum_{b, p} dz[b][co][p] x[b][ci][p + (tap - centre) * d],
     db[co] += sum_{b, p} dz[b][co][p]          (ACCUMULATED: zero them first).
   x, dz: C32; dw (FP32 [c_out][c_in][27]) or db may be NULL. The sums over voxels run on the
   tensor cores with FP32 accumulation. */
rt_status rt_conv3d_weight_grad(const void* x, const void* dz, int B, int D, int H, int W, int c_in,
                                int c_out, int dilation, float* dw, float* db, void* cuda_stream);

/* Surrogate input features from FP32 kappa, j [B][D][H][W]: C32 holding
   channel 0 = log(kappa / 0.05), channel 1 = log(1 + j), other channels 0. */
rt_status rt_surrogate_features(const float* kappa, const float* j, int B, int D, int H, int W, void* x,
                                void* cuda_stream);

/* out[b] = max over vox of field[b][vox] (field >= 0). */
rt_status rt_field_max(const float* field, int B, long long vox, float* out, void* cuda_stream);

/* Training loss of the surrogate: *loss += mean over b, v of (pred - T)^2 with the target
   T = (log(field + eps_rel * fmax[b]) - mu) / sigma (the log field, standardised); when grad is
   non-NULL its gradient 2 (pred - T) / (B vox) is written to channel 0 of the C32 tensor grad
   (the other channels 0). pred, field: FP32 [B][vox]. */
rt_status rt_log_field_loss(const float* pred, const float* field, int B, long long vox, const float* fmax,
                            float eps_rel, float mu, float sigma, void* grad, float* loss, void* cuda_stream);

/* Per-field error sums of the surrogate: out[2b] = sum (F' - F)^2, out[2b+1] = sum F^2 with the
   prediction F' = exp(pred sigma + mu) - eps_rel * fmax[b]; out is overwritten. */
rt_status rt_field_error(const float* pred, const float* field, int B, long long vox, const float* fmax,
                         float eps_rel, float mu, float sigma, float* out, void* cuda_stream);

/* out[b][c] = mean over voxels of channel c < C of a C32 tensor (overwritten). */
rt_status rt_c32_channel_mean(const void* x, int B, int C, long long vox, float* out, void* cuda_stream);

/* One bias-corrected Adam step on n FP32 parameters (step >= 1 counts from 1). */
rt_status rt_adam_step(float* params, const float* grads, float* m, float* v, long long n, float lr,
                       float beta1, float beta2, float eps, int step, void* cuda_stream);

/* Synchronising read-and-clear of this device's kernel error word: RT_OK, or RT_ERR_TIMEOUT
   with *code = which wait gave up (1-4, 11: convolution ring / accumulator / completion, 5-9:
   weight gradient, 10: shared memory not 1024-byte aligned). */
rt_status rt_device_status(int* code);

/* Synchronise the stream (NULL: legacy default stream) and report what the device left:
   RT_ERR_CUDA with the CUDA error's text if one is pending, RT_ERR_TIMEOUT if a kernel with
   bounded waits gave up (as rt_device_status, whose word it clears), else RT_OK. */
rt_status rt_sync_status(void* cuda_stream);

/* ---- Microbenchmarks (no counterpart in the paper) ----------------------------------
   Peaks of the memory operations the march is built from, measured on the current device so
   the march's roofline fractions have a denominator from the same GPU. One launch of
   8 x (SM count) blocks of 256 threads, each thread doing `iters` operations on the device
   buffer `buf` (buf_bytes bytes, contents overwritten; keep it L2-resident, e.g. 32 MiB):
     kind 0: red.global.add.f32 (vec 1) / .v4.f32 (vec 4) into uniformly random vectors;
     kind 1: the same, each warp on 32 consecutive vectors at a random position;
     kind 2: the same into the 8 corners of a random cell of an edge^3 grid of vectors
             (cell-major, the march's packed accumulator layout; 8 operations per iteration);
     kind 3: read-only loads of uniformly random vectors;
     kind 4: read-only loads of the 8 corners of a random cell of an edge^3 grid;
     kinds 5 / 6: kind 2 with 8-byte cells, red.global.add.u64 (the fixed-point deposit) /
             red.global.add.f64 (vec must be 1).
   Addresses come from a per-thread linear congruential generator and are in bounds by
   construction. *ms = device time of the launch (CUDA events on the legacy default stream; the
   call synchronises), *ops = vector operations performed. Errors: RT_ERR_INVALID_ARG for a bad
   kind / vec / iters (1 .. 2^20), a NULL pointer, a buffer of fewer than 32 vectors (kinds 0,
   1, 3) or one that does not hold edge^3 vectors (kinds 2, 4, 5, 6; 2 <= edge <= 2048). */
rt_status rt_microbench(int kind, int vec, void* buf, long long buf_bytes, int edge, int iters, float* ms,
                        double* ops);

/* The attenuation factor exp(-x) exactly as every march kernel computes it (2^(-x log2 e) on
   the device's base-2 exponential, subnormal results flushed to zero), for n device values:
   y[i] = exp(-x[i]). x and y are device arrays of n floats (caller-owned, may not overlap
   partially; y = x is allowed), enqueued on `stream` (NULL: legacy default stream), no
   synchronisation. For checking the factor's accuracy. Errors: RT_ERR_INVALID_ARG for n < 0 or
   a NULL array with n > 0; RT_ERR_CUDA if the launch fails. */
rt_status rt_neg_exp(const float* x, float* y, long long n, void* stream);

/* Launch plan of the last forward call on this handle: bin-group width (1, 2 or 4 bins per
   group), threads per block, gather mode (0: reuse, 1: ahead, 2: both), lanes per ray, source
   deposit tiles (0 / 1), and the march time the autotuner measured for it in ms (-1 when
   rt_options.autotune is 0). Any pointer may be NULL.
   With autotune = 1, the first call of each shape class (n_freq, num_sources, rays, N_s)
   times every candidate plan on its own inputs before running; it synchronises the stream. */
rt_status rt_last_plan(rt_grid* grid, int* width, int* block, int* prefetch, int* lanes_per_ray, int* tile,
                       float* tuned_ms);

/* Multi-device partition of one advance (Sec. 2: the directions are sharded across devices,
   each device sums its part, and one reduction across devices combines them; here the
   (source, ray) pairs are split, which removes the paper's need for N_Omega divisible by the
   device count). Host only, no device call. Shard `shard` of `n_shards` owns a contiguous range
   of the source-major (source, ray) pairs; range sizes differ by at most one pair. The range is
   written as *n_pieces <= 3 pieces to HOST pieces[4 * i + 0..3] = (source_begin, source_end,
   ray_begin, ray_end): march each with rt_advance_rays on sources [source_begin, source_end)
   (pointer source_pos + 3 * source_begin) and rays [ray_begin, ray_end) of the num_rays lattice,
   the first piece overwriting the shard's partial field and the others accumulating; the sum of
   all shards' partial fields is rt_advance's field. An empty shard (fewer pairs than shards)
   has no piece. RT_ERR_INVALID_ARG for num_sources < 0, num_rays < 1 or shard outside
   [0, n_shards). */
rt_status rt_shard_plan(int num_sources, int num_rays, int n_shards, int shard, int* pieces, int* n_pieces);

/* Checkpoint stride K of the last rt_backward* on this handle, and the reverse-march time in ms
   the stride tuner measured for it (-1 when it was not tuned). Either pointer may be NULL. */
rt_status rt_last_ckpt_stride(rt_grid* grid, int* stride, float* tuned_ms);

/* Accumulation of the last forward call on this handle: *mode = 1 FP32 reductions, 2 FP64
   reductions, 3 64-bit fixed point (deterministic mode). */
rt_status rt_last_accumulation(rt_grid* grid, int* mode);

/* Text of the last autotuning pass on this handle: one line per candidate plan with its best
   march time ("W=4 block=64 prefetch=0 lanes=2 0.5123 ms"), copied NUL-terminated into the HOST
   buffer buf of len bytes (truncated if needed; "" if the handle never tuned). */
rt_status rt_tuning_report(rt_grid* grid, char* buf, int len);

/* Test hook: per-substep cell indices of lattice ray `ray` from the HOST position src[3]
   on this handle's grid, computed on the device by the march's own geometry code.
   base_cell[k] = flat index of the clamped floor corner of x_k; kappa_cell[k] = flat index
   of the kappa cell (rt_options.kappa_mode). Host outputs of num_steps entries each.
   Synchronous. */
rt_status rt_trace_cells(rt_grid* grid, const float* src, int num_rays, int ray, float step_size,
                         int num_steps, long long* base_cell, long long* kappa_cell);

#ifdef __cplusplus
}
#endif

#endif /* RAYTRAX_H */
