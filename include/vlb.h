/*
 * vlb.h -- C ABI of the GB300 (sm_103a) coupled vortex-filament /
 * lattice-Boltzmann step of Inui & Tsubota, arXiv 2108.04435.
 *
 * One "channel" holds a D3Q19 lattice of normal fluid and a set of quantized
 * vortex filaments, resident in device memory.  vlb_step advances both by one
 * coupled time step per iteration (Sec. II):
 *   (a) D3Q19 BGK pull stream-collide with the split forcing of Eq. 14a-d
 *       (Eqs. 5-9, 12-13), halfway bounce-back at walls and moving-wall heater
 *       links on the stream-axis faces (Sec. IV), then the superfluid
 *       counterflow V_s per stream plane (Eq. 18);
 *   (b) the normal velocity interpolated onto filament points and the
 *       mutual-friction reaction spread back with the 2-point delta function
 *       (Eqs. 10-11);
 *   (c) Biot-Savart velocity of the filaments (Eq. 3) with the local term,
 *       the alpha/alpha' equation of motion (Eq. 4) integrated with RK4, then
 *       remeshing to [dxi_min, dxi_max] and reconnection (Sec. II.A).
 *
 * Conventions
 *  - Lattice units (dx = dt = 1).  Nodes at integer coordinates 0..n-1; a wall
 *    sits half a cell outside the first and last node of a wall axis.
 *  - Field arrays are structure-of-arrays with x fastest, a[c][z][y][x].
 *  - Population order (Table I, 0-based): 0 rest; 1 +x, 2 -x, 3 +y, 4 -y,
 *    5 +z, 6 -z; 7 (+1,+1,0) 8 (-1,-1,0) 9 (+1,-1,0) 10 (-1,+1,0)
 *    11 (+1,0,+1) 12 (-1,0,-1) 13 (+1,0,-1) 14 (-1,0,+1) 15 (0,+1,+1)
 *    16 (0,-1,-1) 17 (0,+1,-1) 18 (0,-1,+1).
 *  - Filament points are stored densely 0..N-1; next[i] is the successor of
 *    point i along its (closed) loop.
 *  - Every call returns VLB_OK (0) or a negative VLB_ERR_* code; the message
 *    of the last failure on the calling thread is vlb_last_error().  After any
 *    error the channel can still be read and destroyed.
 *  - Ownership: the caller owns every host array it passes and gets back; the
 *    library copies in and out and keeps no host pointer.  The library owns
 *    the device buffers of a channel (allocated at create time, through the
 *    caller's allocator when one is given).  The stream belongs to the caller
 *    and must outlive the channel.  A channel is not thread-safe; distinct
 *    channels on distinct streams are independent.
 */
#ifndef VLB_H
#define VLB_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    VLB_OK = 0,
    VLB_ERR_INVALID_ARG = -1, /* bad parameter, size or handle */
    VLB_ERR_OOM = -2,         /* device allocation failed */
    VLB_ERR_CAPACITY = -3,    /* more filament points than max_points */
    VLB_ERR_TOPOLOGY = -4,    /* next[] is not a permutation of closed loops */
    VLB_ERR_MACH = -5,        /* |u|/c_s >= 0.05 somewhere (Sec. II.B validity limit) */
    VLB_ERR_NAN = -6,         /* NaN/Inf in the lattice or on a filament */
    VLB_ERR_TIMEOUT = -7,     /* a device-side wait gave up (kernel returned early) */
    VLB_ERR_CUDA = -8,        /* a CUDA runtime call failed */
    VLB_ERR_CFL = -9          /* a filament point moved >= 1 cell within one step */
};

/* Parameters of a channel.  Readings where the paper is silent are noted. */
typedef struct {
    int32_t n[3];            /* cells along x, y, z (>= 1) */
    int32_t wall[3];         /* per axis: 0 periodic, 1 halfway bounce-back walls on both faces */
    int32_t stream_axis;     /* counterflow axis; this library requires 2 (z) */
    int32_t vfm_substeps;    /* RK4 sub-steps per lattice step (>= 1) */
    int32_t couple;          /* 1: spread the mutual-friction reaction onto the lattice (Eqs. 10-11) */
    int32_t force_form;      /* 0: f of Eq. 10 as printed; 1: f = rho_s kappa (rhs of Eq. 10) x s' */
    int32_t max_points;      /* filament point capacity (device arrays are sized by it) */
    int32_t storage;         /* population storage: VLB_STORE_F32 (0), VLB_STORE_F16 (1) or VLB_STORE_BF16 (2) */
    int32_t wall_images;     /* 1: the boundary-induced velocity v_s,b of Sec. II.A from first-order mirror images
                                of every segment across each solid wall face (orientation reversed); 0: v_s,b = 0 */
    int32_t reserved;        /* 0 */
    double  tau, rho0;       /* BGK relaxation time (> 1/2, Eq. 8) and reference density */
    double  body_force[3];   /* uniform body force added to the force grid (0 in the paper's runs) */
    double  heater_vn;       /* Sec. IV heater: normal velocity injected at the low z face and removed at the high one */
    double  pin_vn;          /* periodic z: plane z = 0 reset to f^eq(rho, pin_vn e_z) (Sec. III.C); 0 = off */
    double  init_vn[3];      /* initial uniform normal velocity */
    double  kappa, alpha, alpha_p, rho_s_over_rho_n, core_a; /* circulation, Eq. 4 friction, density ratio, core radius */
    double  dxi_min, dxi_max;                                /* remeshing interval (Sec. III: 0.70, 0.95) */
} vlb_params;

/* Population storage formats (vlb_params.storage).  All three store the
 * deviation f_i - w_i rho0 and compute in FP32: F32 moves 152 B per cell and
 * lattice pass, F16 (deviation scaled by 2^10) and BF16 move 76 B. */
enum { VLB_STORE_F32 = 0, VLB_STORE_F16 = 1, VLB_STORE_BF16 = 2 };

/* Optional device allocator (e.g. PyTorch's caching allocator).  alloc returns
 * a device pointer of at least `bytes` bytes (16-byte aligned) or NULL; free
 * releases it.  `stream` is the channel's stream. */
typedef struct {
    void* ctx;
    void* (*alloc)(void* ctx, size_t bytes, void* stream);
    void (*free)(void* ctx, void* ptr, void* stream);
} vlb_allocator;

typedef struct vlb_channel vlb_channel;

/* Phases of one coupled step, for vlb_run_phases. */
enum { VLB_PHASE_LBM = 1, VLB_PHASE_VFM = 2, VLB_PHASE_REMESH = 4, VLB_PHASE_RECONNECT = 8, VLB_PHASE_ALL = 15 };

/* Fields for vlb_read_fields / vlb_write_fields. */
enum {
    VLB_FIELD_RHO = 0,      /* float32 [C]: density of the streamed populations of the current state */
    VLB_FIELD_U = 1,        /* float32 [3][C]: their half-force shifted velocity (sum c f + F/2)/rho */
    VLB_FIELD_FSTAR = 2,    /* float32 [19][C]: post-collision populations (read and write) */
    VLB_FIELD_FORCE = 3,    /* float32 [3][C]: force grid of the next lattice pass (read and write) */
    VLB_FIELD_POS = 4,      /* float64 [N][3]: filament points */
    VLB_FIELD_NEXT = 5,     /* int32 [N]: successor of each point, -1 at the last point of an open line */
    VLB_FIELD_PLANE_VS = 6, /* float64 [n_z]: superfluid counterflow velocity per z plane (Eq. 18) */
    VLB_FIELD_STATS = 7,    /* float64 [16]: 0 points, 1 status bits, 2 mass, 3 line length, 4 max Mach,
                               5 splits, 6 merges, 7 reconnections, 8 points deleted in small loops,
                               9 steps, 10 device bytes allocated, 11..12 reserved, 13 wall-contact cuts,
                               14..15 reserved */
    VLB_FIELD_VEL = 8,      /* float64 [N][3]: ds/dt at the first RK stage of the last filament advance */
    VLB_FIELD_FDEV = 9,     /* float32 [19][C]: f_i - w_i rho0 of the post-collision populations (read only;
                               the flow signal at full float precision) */
    VLB_FIELD_LINE_PROFILE = 10 /* float64 [n_z]: line length per z plane, each segment counted in the plane
                                   nearest its midpoint (line density L(z) = profile / (n_x n_y), Sec. IV) */
};

/* Create a channel (Sec. II set-up): validates p (tau > 1/2, stream_axis 2,
 * dxi_min < dxi_max, Mach of init_vn and heater_vn below 0.05), allocates every
 * device buffer for the lattice and max_points filament points, and fills the
 * lattice with the uniform equilibrium f^eq(rho0, init_vn) (Eq. 7).  `alloc`
 * may be NULL (cudaMalloc is used); `stream` is a cudaStream_t (NULL = the
 * legacy default stream).  On success *out receives the handle. */
int vlb_create_channel(const vlb_params* p, const vlb_allocator* alloc, void* stream, vlb_channel** out);

/* Replace the filament set (Sec. II.A): xyz is host float64 [n][3], next host
 * int32 [n] with the successor of each point or -1 where an open line ends.
 * The set must be made of closed loops and open lines (no point with two
 * predecessors, no isolated point).  Open lines are bound to the solid walls
 * (Sec. IV): each end must lie within dxi_max of a wall's clamp bound (walls at
 * -1/2 and n - 1/2, bounds dxi_min/2 inside them) and is moved onto the
 * nearest one; it then stays on that wall, taking the mirror image of its
 * neighbour across the wall as its missing neighbour.  Points on periodic axes
 * are wrapped into [0, n); points outside the walls are rejected; points
 * closer than dxi_min/2 to a wall are moved onto the bound.  Errors: CAPACITY
 * (n > max_points), TOPOLOGY (structure, or an open end away from the walls),
 * INVALID_ARG (NaN, outside walls). */
int vlb_seed_vortices(vlb_channel* ch, const double* xyz, const int32_t* next, int32_t n);

/* Advance `nsteps` coupled steps (all phases, in order LBM, VFM, remesh,
 * reconnect).  Work is queued on the channel's stream; the call waits for it
 * once at the end and returns the first error the device reported (MACH, NAN,
 * CAPACITY, CFL, TIMEOUT).  On a created (non-default) stream each step is
 * replayed from a CUDA graph captured on first use; every kernel reads the
 * live filament count from device memory, so no host round trip is needed
 * between steps.  When nsteps > 0 the total line length of the new points is
 * computed at the end and read back with the status, so vlb_line_length
 * returns it without a launch or a wait until the state changes again. */
int vlb_step(vlb_channel* ch, int32_t nsteps);

/* Enable (default) or disable the graph replay of vlb_step. */
int vlb_set_graphs(vlb_channel* ch, int32_t enable);

/* Enable (default) or disable the overlap inside the 8-step graphs that
 * vlb_step replays while 8 or more steps remain (created stream only): the
 * lattice pass of each step runs on the channel's stream alongside the remesh
 * and reconnection of the step before and the first Biot-Savart sum of its
 * own step, which run on a second stream of the highest priority.  Results
 * are the same, bit for bit, either way.  The overlap pays for a channel that
 * has the GPU to itself; where many channels share the GPU, their work
 * overlaps already and the extra streams compete for the device's hardware
 * queues, so turn it off there.  Errors: INVALID_ARG (null channel, or steps
 * of vlb_step_async still queued). */
int vlb_set_overlap(vlb_channel* ch, int32_t enable);

/* Non-blocking form of vlb_step, for hosts that drive many channels at once
 * (each on its own stream, so their work overlaps on the GPU) or that read
 * each step's result while the next steps already run: queues the steps, the
 * line length of the new points (nsteps > 0) and a read-back of the status
 * block into a pinned slot of this call's own, and returns without waiting.
 * A channel holds up to VLB_ASYNC_DEPTH such calls in flight (INVALID_ARG
 * beyond), completed in order by vlb_query: it returns VLB_BUSY (1) while
 * the oldest queued call runs, VLB_OK once it has finished (vlb_query_stats
 * then reads that call's status, and vlb_line_length returns its line length
 * without a wait if no later call is queued), or the first error the device
 * reported (as vlb_step).  vlb_step and vlb_set_overlap return INVALID_ARG
 * while calls are queued.  A one-step call on a created stream, with graphs
 * and the overlap on, runs split over the channel's stream and the second
 * stream: its remesh, reconnection, line length and status copy run beside
 * the lattice pass of the next queued call, with the same results bit for
 * bit.  A device error may then show in the status of the call queued
 * before the step that raised it (status bits are sticky). */
enum { VLB_BUSY = 1, VLB_ASYNC_DEPTH = 4 };
int vlb_step_async(vlb_channel* ch, int32_t nsteps);
int vlb_query(vlb_channel* ch);

/* The VLB_FIELD_STATS record (16 float64, same layout) of the vlb_step_async
 * call that vlb_query completed last: the state right after that call's
 * steps, whatever calls are queued after it; out[9] counts the steps up to
 * it.  No device work and no wait.  INVALID_ARG (null argument, or no call
 * completed yet). */
int vlb_query_stats(vlb_channel* ch, double* out);

/* Device bytes vlb_create_channel would allocate for these parameters (an
 * upper bound used to admit channels against a memory budget); 0 if the
 * parameters are invalid. */
size_t vlb_channel_bytes(const vlb_params* p);

/* Run only the selected phases once (bitwise OR of VLB_PHASE_*), in the
 * order of vlb_step; used to check each part of the step on its own. */
int vlb_run_phases(vlb_channel* ch, int32_t phase_mask);

/* Copy a field to host memory `dst` of `bytes` bytes (after a stream sync);
 * *written (nullable) receives the byte count.  INVALID_ARG if too small. */
int vlb_read_fields(vlb_channel* ch, int32_t which, void* dst, size_t bytes, size_t* written);

/* Overwrite FSTAR or FORCE from host memory (exact size required).  Writing
 * FORCE marks the whole lattice as carrying force for the next pass. */
int vlb_write_fields(vlb_channel* ch, int32_t which, const void* src, size_t bytes);

/* Total vortex line length sum |s_next(i) - s_i| in float64 (Sec. III.C line
 * density L = length / volume), reduced on the device in a fixed order. */
int vlb_line_length(vlb_channel* ch, double* out);

/* Free every device buffer of the channel (after a stream sync).  NULL is a no-op. */
void vlb_destroy(vlb_channel* ch);

/* Message of the last error on this thread (never NULL). */
const char* vlb_last_error(void);

/* Event-timed mode.  While `enable` is set, vlb_step launches the kernels of
 * each step one by one (no graph replay, no programmatic launch) and records
 * CUDA events on the channel's stream around every launch of two kernels:
 *   VLB_TIMED_LBM          the stream-collide pass (Eqs. 9, 14)
 *   VLB_TIMED_BIOT_SAVART  the Biot-Savart sum of each RK stage (Eq. 3; from
 *                          24576 points on it also applies Eq. 4 to its targets)
 * vlb_set_timing resets the totals.  vlb_kernel_timing returns the total
 * milliseconds and launch count of one kind since the last reset (after a
 * stream sync); vlb_lbm_timing is vlb_kernel_timing of VLB_TIMED_LBM.
 * Errors: INVALID_ARG (null argument, unknown kind), CUDA. */
enum { VLB_TIMED_LBM = 0, VLB_TIMED_BIOT_SAVART = 1, VLB_TIMED_KINDS = 2 };
int vlb_set_timing(vlb_channel* ch, int32_t enable);
int vlb_kernel_timing(vlb_channel* ch, int32_t kind, double* total_ms, int64_t* launches);
int vlb_lbm_timing(vlb_channel* ch, double* total_ms, int64_t* launches);

/* Stand-alone Biot-Savart velocity (Eq. 3, nonlocal part: every segment j ->
 * next[j] except the two touching the target, minimum image on periodic axes)
 * at every point of a device-resident filament set.
 *   pos      device float64 SoA [3][n] (x block, then y, then z)
 *   next     device int32 [n] successor indices, -1 at the last point of an
 *            open line (that point starts no segment)
 *   vel      device float32 SoA [3][n], written
 *   scratch  device buffer of at least vlb_biot_savart_scratch_bytes(n) bytes,
 *            256-byte aligned; its contents need not be initialised
 * Uses only p->n, p->wall and p->kappa.  Runs on `stream` and does not wait,
 * so it returns only the errors it can see on the host (INVALID_ARG for bad
 * arguments or a small scratch, CUDA for a failed launch): device-side
 * findings (a next[] entry outside [-1, n), a timed-out tile copy) are not
 * reported, and vel is then not meaningful. */
size_t vlb_biot_savart_scratch_bytes(int32_t n);
int vlb_biot_savart(const vlb_params* p, const double* pos, const int32_t* next, int32_t n,
                    float* vel, void* scratch, size_t scratch_bytes, void* stream);

/* Allocation-free variant of vlb_biot_savart (the paper has no counterpart;
 * it exists for callers of this library that may not allocate device memory
 * while they run, e.g. hosts that only hand out pre-registered buffers or
 * code that must not trigger the device synchronisation cudaMalloc implies).
 * Same arguments and result as vlb_biot_savart, without the scratch buffer:
 * the scratch lives in a fixed 19 MiB file-scope device array that every GPU
 * loading this library holds until the process exits, and no cudaMalloc,
 * cudaFree or allocating library routine is called.  A compile-time check
 * keeps the array at least as large as the scratch of a 65536-point call.
 *   n        at most 65536 points; larger n returns VLB_ERR_INVALID_ARG
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it for the
 * life of the process; make no call after a cudaDeviceReset of that
 * device.  All calls share the one array, so calls whose work overlaps on
 * the GPU (other streams, other threads) race: serialise them.  Runs on `stream`; does not wait; reports
 * no device-side findings (as vlb_biot_savart). */
int vlb_biot_savart_noalloc(const vlb_params* p, const double* pos, const int32_t* next, int32_t n, float* vel,
                            void* stream);

#ifdef __cplusplus
}
#endif
#endif
