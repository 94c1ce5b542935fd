// Internal declarations shared by the CUDA translation units of libvlb.
#pragma once
#include <cuda_runtime.h>

#include <utility>
#include <stdint.h>

#include "../../include/vlb.h"

namespace vlb {

// Device status bits, OR-ed by kernels into Dev::counters[CNT_STATUS].
enum : int {
    ST_MACH = 1,
    ST_NAN = 2,
    ST_CAPACITY = 4,
    ST_TIMEOUT = 8,
    ST_CFL = 16,
    ST_TOPOLOGY = 32,  // a successor index outside the live range (never expected)
};

// Device integer counters (one int array).
enum : int {
    CNT_N = 0,          // live filament points
    CNT_TOTAL = 1,      // points before compaction (old + appended)
    CNT_STATUS = 2,     // status bits
    CNT_NPAIRS = 3,     // candidate reconnections this pass
    CNT_STAMP = 4,      // reconnection pass counter (claim stamps)
    CNT_SMALL = 5,      // points deleted in small loops this pass
    CNT_BSWORK = 6,     // Biot-Savart work-item counter (reset before each launch)
    CNT_PLANES = 7,     // z planes reduced in the current lattice pass
    CNT_LINEDONE = 8,   // blocks done in the line-length reduction
    CNT_NCONTACT = 9,   // wall-contact candidates of the current reconnection pass
    CNT_DIRTY = 10,     // 1 after seeding: the next remesh checks for small components even without removals
    CNT_RFLAGS = 11,    // nonzero when the remesh geometry flagged a split or removal candidate (cleared by the finish)
    CNT_NSLOT = 12,     // Biot-Savart source slots of the current step (points + gap slots)
    CNT_PASS = 13,      // 1 when the last topology finish changed nothing: the pass kernel copies the points
    CNT_COUNT = 14
};

// Device float64 statistics.
enum : int {
    DS_MASS = 0,
    DS_MAXMACH = 1,
    DS_LINE = 2,
    DS_SPLITS = 3,
    DS_MERGES = 4,
    DS_RECON = 5,
    DS_SMALL = 6,
    DS_WALLCUT = 7,
    DS_LAT = 8,  // mass and max Mach of the lattice passes of split async steps, one pair per population parity
    DS_COUNT = 12
};

// Stored population formats (vlb_params::storage).
enum : int { STORE_F32 = 0, STORE_F16 = 1, STORE_BF16 = 2 };

constexpr int TILE_SHIFT = 3;   // force / velocity activity tiles of 8^3 cells

// The force grid accumulates the spreading of Eqs. 10-11 in fixed point:
// int64 with FORCE_FRAC fractional bits (resolution 5.7e-14, range 5e5), so
// the atomic additions are exact and their order does not matter; every run
// is bitwise reproducible.  A contribution is rounded to the grid once.
constexpr int FORCE_FRAC = 44;
__device__ __forceinline__ long long force_fixed(float v) { return __float2ll_rn(v * 0x1p44f); }
// The grid value as a float from its two 32-bit words: the high word is exact
// in FP32 while |a| < 2^56 (|F| < 4096), so the result carries at most two
// roundings (the low word, the fused add) instead of one.  A 64-bit integer
// conversion would run on GB300's FP64 pipe, which measured 22% busy in the
// stream-collide pass from these conversions alone.
__device__ __forceinline__ float force_value(long long a) {
    const float hi = __int2float_rn((int)(a >> 32));
    const float lo = __uint2float_rn((unsigned)(a & 0xffffffffll));
    return fmaf(hi, 0x1p32f, lo) * 0x1p-44f;
}

// Biot-Savart split sums below the fused size, accumulated the same way: int64
// with 40 fractional bits (resolution 9.1e-13, range 8.4e6 in lattice units),
// so the sum over splits is exact and independent of their order.
__device__ __forceinline__ long long bs_fixed(float v) { return __float2ll_rn(v * 0x1p40f); }
__device__ __forceinline__ float bs_value(long long a) { return __ll2float_rn(a) * 0x1p-40f; }

// Programmatic dependent launch: the kernels of a step are launched with
// programmatic stream serialisation, so each one is scheduled while its
// predecessor drains.  Every such kernel first waits for its predecessor's
// completion and memory flush (griddepcontrol.wait, a no-op without a
// programmatic predecessor), then lets its own successor be scheduled.
__device__ __forceinline__ void pdl_wait_trigger() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// VLB_PDL=0 in the environment turns programmatic launch off (default on).  It
// is not used while tl_no_pdl is set on this thread: during graph capture (the
// graph schedules its kernel nodes back to back by itself, and measured slower
// with programmatic edges) and in the event-timed mode (an event between two
// kernels must see the first one finished).
bool pdl_enabled();
extern thread_local bool tl_no_pdl;

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = (pdl_enabled() && !tl_no_pdl) ? 1 : 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
constexpr int LBM_BLOCK = 256;  // cells per stream-collide block (one z plane)
constexpr int BS_TPB = 128;     // threads per Biot-Savart block
constexpr int BS_TILE = 128;    // source slots per shared-memory tile
constexpr int BS_GROUP = 64;    // source slots that share one integer origin
constexpr int BS_REC = 5;       // float4 per source slot (80 bytes; slots are stored in interleaved pairs)
constexpr int BS_VALS = 4 * BS_REC;  // values per slot
constexpr int BS_PAIR = 2 * BS_REC;  // float4 per pair of slots
constexpr int MAX_SPLIT = 64;   // Biot-Savart source splits
// From this many points on the Biot-Savart sources are put in a spatial order
// once per step, so that a group of BS_GROUP slots spans a small box
constexpr int BS_SORT_MIN = 8192;
constexpr int BS_SORT_MAX_BINS = 256;  // bins of the spatial order (a key of at most 8 bits)

// Biot-Savart sources as a chain of slots.  Each point of the order
// (sorted position k) owns one slot, slot[k], holding its segment
// s_i -> s_next(i).  The slot after it holds the segment's end point: the
// next point of the order when that is next(i) (the usual case: a line runs
// through a bin as consecutive points), otherwise a gap slot inserted there
// that holds a copy of s_next(i) and no segment.  A line's last point has no
// segment and needs no gap.  So the pair sum can take |R| at a slot's point
// as both the start of its own segment and the end of the one before, one
// reciprocal square root per slot instead of two per segment.
//
// Slot record: 20 values relative to the integer origin O of its group of
// BS_GROUP slots (at the step's start, the integer cell nearest the centre
// of the group's box):
//   0-2 h = fl(s - O) (minimum image on periodic axes), 3 |d|^2, 4-6 d,
//   7-9 c = h x d (FP32), 10-12 l = fl(s - O - h), 13-15 fl(s - O + d), the
//   segment's end (read for the group's last slot, whose end lies in the
//   next group); slots 0 and 1 hold there instead the low and high corner
//   of the group's box of h (unbounded when the chain jumps by a periodic
//   box somewhere in the group); 16 |h|^2 (FP32), 17-19 zero;
// h + l carries s - O to ~1e-14 cells.  Gap and padding slots have d = 0.
// Storage: slot p and slot p + 32 of a group form pair p, interleaved in
// 160 bytes: value v of slot k is float
//   (k / 64) * 1280 + (k % 32) * 40 + 2 v + (k / 32) % 2,
// so that one float4 holds two values of both slots, one float2 the same
// value of both (the packed FP32 pair path), and the pairs p = 0..31 of a
// group walk its two halves along their chains side by side.
// A target r (its own slot: origin O_t, parts h_t, l_t) sees the group at
// offset t = (O - O_t) - h_t - l_t, so R1 = s - r = h + l + t.
__host__ __device__ inline long long bs_value_index(long long k, int v) {
    return (k >> 6) * (BS_GROUP * BS_VALS) + (k & 31) * (2 * BS_VALS) + 2 * v + ((k >> 5) & 1);
}

// Order of the Biot-Savart sources.  sorted = 0: sorted position k is
// point k; sorted = 1: it is point ord[k] (rank is the inverse), a spatial
// order.  slot[k] is the slot of sorted position k, and pt[s] what slot s
// holds: point i >= 0 (its own slot), -2 - i (a gap slot, holding the
// successor of point i) or -1 (padding).  Group g of BS_GROUP slots has the
// integer origin org[g].xyz.  tgt[4k .. 4k + 3] is the target record of
// sorted position k: its slot's parts h, l, origin O (as floats), its slot,
// its predecessor's slot, the excluded image slot of a pinned end, and its
// point index (ints by bit pattern).
struct BsOrder {
    int sorted;
    const int* ord;
    const int* rank;
    const int* slot;
    int* pt;
    int4* org;
    float4* tgt;
};

// Bins of the spatial order: the cell floor(x) >> shift per axis, clamped to
// the lattice, interleaved bit by bit (x, y, z) into a Morton key < K.
// The bin edge is the widest of 64, 32 and 16 cells that still leaves at
// least 64 bins: wider bins break the lines less often (a gap slot wherever
// a line leaves its bin: 1.14 slots per point with 8-cell bins on the
// 128x128x1024 channel, 1.08 with 16, 1.045 with 32, 1.025 with 64), and
// enough bins keep each group of slots compact.  Measured per Biot-Savart
// launch on GB300: the channel 5.71 ms with 16-cell bins, 5.56 with 32, 5.50
// with 64 (64 bins); the 128^3 box 613, 603 and 648 us (8 bins at 64).
// Lattices that would need more than 256 bins widen them further, so that a
// key has at most 8 bits (the counting sort keeps a count per bin for each
// block of points in shared memory).
struct BsBins {
    int shift;
    int bits[3];
    int K;
};

__host__ __device__ inline int bs_ceil_log2(int v) {
    int b = 0;
    while ((1 << b) < v) ++b;
    return b;
}

__host__ __device__ inline BsBins bs_bins(int nx, int ny, int nz) {
    BsBins b;
    auto bins = [&](int sh) {
        const int e = 1 << sh;
        return (long long)((nx + e - 1) / e) * ((ny + e - 1) / e) * ((nz + e - 1) / e);
    };
    b.shift = 6;
    while (b.shift > 4 && bins(b.shift) < 64) --b.shift;
    while (true) {
        const int e = 1 << b.shift;
        b.bits[0] = bs_ceil_log2((nx + e - 1) / e);
        b.bits[1] = bs_ceil_log2((ny + e - 1) / e);
        b.bits[2] = bs_ceil_log2((nz + e - 1) / e);
        const int tot = b.bits[0] + b.bits[1] + b.bits[2];
        if (tot <= 8) {
            b.K = 1 << tot;
            return b;
        }
        ++b.shift;
    }
}

// Slots of one block of sources (the segments, or their images across one
// wall) for ns slots: whole groups, the padding slots zero.
__host__ __device__ inline long long bs_block(int ns) { return (long long)((ns + BS_GROUP - 1) / BS_GROUP) * BS_GROUP; }
// Slot capacity for up to n points: every point may need a gap slot.
__host__ __device__ constexpr long long bs_slot_cap(long long n) { return ((2 * n + BS_GROUP - 1) / BS_GROUP) * BS_GROUP; }
// Blocks of the slot scan (each takes a contiguous range of sorted positions).
constexpr int BS_SLOT_BLOCKS = 256;

// Geometry of the lattice, passed by value to kernels.
struct Grid {
    int nx, ny, nz;
    int wall[3];
    long long ncell;
    int tnx, tny, tnz;  // activity tiles per axis
};

// Flag the velocity tiles within one cell of point x (the nodes the 2-point
// delta function of Eq. 11 can reach, with a cell of margin): the
// stream-collide pass writes u only in flagged tiles.
__device__ __forceinline__ void mark_velocity_tiles(const Grid& g, double x, double y, double z,
                                                    uint8_t* __restrict__ umask) {
    const int n[3] = {g.nx, g.ny, g.nz};
    const double xs[3] = {x, y, z};
    int t[3][4];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int b = (int)floor(xs[a]);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int c = b - 1 + k;
            if (g.wall[a]) c = c < 0 ? 0 : (c > n[a] - 1 ? n[a] - 1 : c);
            else c = ((c % n[a]) + n[a]) % n[a];
            t[a][k] = c >> TILE_SHIFT;
        }
    }
#pragma unroll
    for (int kz = 0; kz < 4; ++kz)
#pragma unroll
        for (int ky = 0; ky < 4; ++ky)
#pragma unroll
            for (int kx = 0; kx < 4; ++kx) umask[(t[2][kz] * g.tny + t[1][ky]) * g.tnx + t[0][kx]] = 1;
}


struct LbmParams {
    Grid g;
    float omega;        // 1/tau
    float pref;         // 1 - 1/(2 tau)
    float rho0;
    float body[3];
    float heater;       // heater_vn
    float pin;          // pin_vn
    float dr0;          // rho0 * (sum_i s_i - 1): density carried by the float shift constants s_i
    float dw[3];        // w_i rho0 - s_i for the rest, axis and diagonal classes (exact in double, then float)
    int body_on;
    int pin_on;
    int vec;            // cells per thread of the stream-collide kernel (4, 2, or 1 = scalar kernel)
    int block;          // threads per block of the scalar kernel (128 or 256)
    int storage;        // STORE_F32, STORE_F16 (deviation x 2^10) or STORE_BF16
    int stream_hint;    // evict-first loads and stores of the populations (one population buffer fits in L2)
    int all_u;          // write v_n in every tile, flagged or not (a pass queued before its points exist)
    unsigned long long nx_magic;  // y = (xy * nx_magic) >> nx_shift equals xy / nx for 0 <= xy < nx * ny
    int nx_shift;
    double inv_ratio;   // rho_n / rho_s
    // device buffers of the fused per-plane reduction (Eq. 18, mass, Mach)
    int* plane_ticket;  // [nz] blocks done per plane, back to 0 after the plane is reduced
    double* plane;      // [nz][3] plane sums (delta rho, u_z, max u^2)
    double* Vs;         // [nz]
    double* dstats;
    int* counters;
};

struct VfmParams {
    Grid g;
    double kappa, alpha, alpha_p, ratio, rho0, core_a, dmin, dmax;
    double dt;
    float kq_f;      // kappa / (4 pi)
    float beta_c_f;  // ln(2 / (e^{1/4} a)), the constant part of the local coefficient
    float alpha_f, alpha_p_f;
    float gscale_f;  // -(rho_s/rho_n) rho0 kappa
    int couple, force_form;
    // wall images (v_s,b): the solid faces, as wall codes 2*axis + side, whose
    // mirror images of the segments are Biot-Savart sources; 0 faces = v_s,b off
    int nfaces;
    int face_code[6];
};

// Arguments of the equation of motion at one RK4 stage (eom.cuh).
struct EomArgs {
    VfmParams P;
    int stage, spread, cap;
    int first;          // the first sub-step of the lattice step (its stage-1 velocity is exported)
    const double* s0;   // RK4 base positions
    double* st;         // stage positions (written for the next stage)
    double* pos_out;    // new positions (last stage)
    double* acc;        // RK4 sum
    double* vel1;       // stage-1 velocity (exported)
    const float4* geo;  // stage geometry
    const float* U;     // v_n grid
    const double* Vs;   // V_s per plane
    long long* F;       // force grid (spreading at stage 0)
    uint8_t* fmask;
    int* counters;
};

// Biot-Savart source splits for N points (targets in tiles of `tile`) and
// `groups` groups of source slots, on a GPU of nsm SMs: about 3 (target
// tile, split) work items per resident block (8 blocks on each SM), taken
// from a device counter, so that the SMs finish together (one item per block
// left a fifth of the SMs idle at the end: 12% slower at 17k and 86k
// points), and at least one group per split (with few points an item is then
// a single group, and the kernel's time is that of one item).  The kernel
// derives it from the device-side counts, so it needs no host estimate.
__host__ __device__ inline int bs_splits(int N, int tile, int nsm, int groups) {
    const int n = N > 0 ? N : 1;
    const int tb = (n + tile - 1) / tile;
    int ns = (3 * 8 * nsm + tb - 1) / tb;
    if (ns > groups) ns = groups;
    if (ns < 1) ns = 1;
    if (ns > MAX_SPLIT) ns = MAX_SPLIT;
    return ns;
}

struct Dev {
    // lattice
    void* f[2];         // stored deviations f_i - s_i, [19][C] in the storage format
    long long* F;       // force grid [3][C], fixed point (FORCE_FRAC fractional bits)
    float* U;           // velocity of the last pass [3][C], valid in u-active tiles
    uint8_t* fmask;     // tiles where F may be non-zero
    uint8_t* umask;     // tiles where U must be written
    float* part;        // stream-collide warp partials [nz][warps per plane][3]
    double* plane;      // plane sums [nz][3]
    int* plane_ticket;  // [nz]
    double* Vs;         // [nz]
    double* dstats;     // [DS_COUNT]
    int* counters;      // [CNT_COUNT]
    // filaments (SoA [3][cap] float64)
    double* pos[2];
    int* next[2];
    int* prev[2];
    double* s0;
    double* st;
    double* acc;
    double* vel1;
    double* spp;        // FP64 curvature for remeshing
    double* seglen;     // FP64 segment lengths for remeshing
    float4* seg;        // Biot-Savart source slots, BS_REC float4 each (segments, then wall images)
    int* bs_key;        // spatial order: Morton key of each point
    int* bs_hist;       // spatial order: per-block bin counts, then their scan
    int* bs_ord;        // sorted position -> point
    int* bs_rank;       // point -> sorted position
    int4* bs_org;       // integer origin of each group of BS_GROUP slots (w: jump flag)
    int* bs_slot;       // sorted position -> slot
    int* bs_pt;         // slot -> its point (or gap, padding) [slot capacity]
    float4* bs_tgt;     // target records, 4 float4 per sorted position
    int* bs_bsum;       // gap slots per block of the slot scan [BS_SLOT_BLOCKS]
    float* bsp;         // Biot-Savart partial sums [splits][3][cap]
    float* vbs;         // Biot-Savart velocity [3][cap]
    long long* vacc;    // Biot-Savart velocity [3][cap], fixed point (bs_fixed), zero between uses
    int* tile_ticket;   // per target tile: splits done
    float4* geo;        // stage geometry: (s', dxi), (local velocity, 0) per point
    // topology scratch
    uint8_t* flags;
    uint8_t* alive;
    int* nnext;
    int* newidx;
    int* hkey;
    int* hhead;         // first point of each hash bucket (-1 empty), kept all -1 between passes
    int* hlink;         // next point in the same bucket
    float4* hpos;       // per point: FP32 position and (as int bits) hlink, read by the nearest-point search
    int* nn;
    double* nd2;
    int* cand_i;
    int* cand_a;
    int* cand_b;
    double* cand_d2;
    int* cand_order;
    int* stamp;
    double* line_part;
};

// ---------------------------------------------------------------- launchers
// lbm.cu
void launch_lbm_init(const LbmParams& P, void* f, float* U, const double init_u[3], cudaStream_t s);
void launch_lbm_step(const LbmParams& P, const void* fin, void* fout, const long long* F, float* U,
                     const uint8_t* fmask, const uint8_t* umask, float* part, cudaStream_t s);
void launch_plane_vs(const LbmParams& P, const float* part, long long* F, uint8_t* umask, uint8_t* fmask,
                     cudaStream_t s);
int lbm_blocks_per_plane(const LbmParams& P);
int lbm_warps_per_plane(const LbmParams& P);
void launch_moments(const LbmParams& P, const void* f, const long long* F, const uint8_t* fmask, float* rho,
                    float* U, cudaStream_t s);
void launch_mark_umask(const Grid& g, const double* pos, const int* counters, int cap, uint8_t* umask,
                       cudaStream_t s);
void launch_zero_force(const Grid& g, long long* F, uint8_t* fmask, cudaStream_t s);
void launch_force_export(const Grid& g, const long long* F, float* out, cudaStream_t s);
void launch_force_import(const Grid& g, const float* in, long long* F, cudaStream_t s);
void launch_export(const LbmParams& P, const void* f, float* out, int i0, int i1, int mode, cudaStream_t s);
void launch_import(const LbmParams& P, const float* in, void* f, int i0, int i1, cudaStream_t s);

// vfm.cu
// The stage geometry writes the Biot-Savart source slots and target records
// of the order `o`, one block per group of slots; span: points one pass
// covers (the groups of 2 span slots; it strides over any beyond).
void launch_geometry_stage(const VfmParams& P, const double* s, const int* next, const int* prev, int* counters,
                           int cap, int span, float4* geo, float4* seg, double* s0_copy, const BsOrder& o,
                           cudaStream_t st);
// vacc != nullptr: the Biot-Savart velocity is read from the fixed-point sums,
// which the kernel clears again for the next pass.
void launch_eom(const EomArgs& A, const float* vbs, cudaStream_t s, long long* vacc = nullptr);
void launch_line_profile(const Grid& g, const double* pos, const int* next, const int* counters, int cap,
                         double* prof, cudaStream_t s);
void launch_line_length(const Grid& g, const double* pos, const int* next, int* counters, int cap, double* part,
                        double* dstats, cudaStream_t s);

// bs.cu
// SMs of the current device (queried once per device).
int sm_count();
int bs_max_splits(int cap, int nsm);
// Spatial order of the points pos[3][cap] (count from the device counters):
// bs_ord and bs_rank.  hist: scratch of at least
// BS_SORT_MAX_BINS * ceil(cap / 1024) ints (at most cap for every cap the
// order is built for).  The grids cover all cap points, so a count that grew
// within the step is ordered whole.
void launch_bs_sort(const Grid& g, const double* pos, int cap, const int* counters, int* key, int* hist, int* ord,
                    int* rank, cudaStream_t s);
// Slots of the order o for the points pos[3][cap] with successors next[]
// (indices outside [-1, N) count as -1): o.slot, o.pt, the group origins
// o.org and counters[CNT_NSLOT].  bsum: scratch [BS_SLOT_BLOCKS].
void launch_bs_slots(const double* pos, const int* next, int cap, int span, int* counters, const BsOrder& o,
                     int* bsum, cudaStream_t s);
// With eom != nullptr the kernel applies the equation of motion to each target
// tile as soon as its sum is complete, and does not write vel.
// Sources are the N segments, then with nfaces > 0 their images across each
// face (records (1 + f) N .. (2 + f) N - 1, written by the stage geometry);
// geo then gives each pinned end's wall, whose image of its own segment is
// left out.
void launch_biot_savart(const Grid& g, double kappa, const float4* seg, const int* prev, const int* counters,
                        int* tile_ticket, int cap, int n_hint, float* part, float* vel, cudaStream_t s,
                        const BsOrder& o, const EomArgs* eom = nullptr, int nfaces = 0,
                        const int* face_code = nullptr, const float4* geo = nullptr, long long* vacc = nullptr);
// Below BS_ACC_MAX points the Biot-Savart split sums go to the fixed-point
// accumulator and a separate kernel applies the equation of motion; from it on,
// the splits write partial sums, the last split of a target tile adds them,
// and (by default) applies the equation of motion in the same kernel.
// Measured per coupled step: at 1.1k points the accumulator made it 6% faster
// than partial sums; at 17k, 1.4% faster than the fused partial-sum kernel;
// at 86k, 3% slower (16M atomic adds per pass).
constexpr int BS_ACC_MAX = 24576;
// Whether launch_biot_savart, given vacc and no equation of motion, adds the
// split sums of about n_hint points into vacc (else it writes vel).
bool bs_uses_vacc(int n_hint);
// Stand-alone entry: prev[], the spatial order (from BS_SORT_MIN points on),
// the slots and the source records of a caller's point set, into the scratch
// buffers.
void launch_bs_standalone_prep(const Grid& g, const double* pos, const int* next, int n, int* prev, float4* seg,
                               int* counters, const BsOrder& o, int* key, int* hist, int* bsum, cudaStream_t s);
// vel[3][n] = the fixed-point sums vacc[3][n] (stand-alone entry)
void launch_bs_unfix(const long long* vacc, int n, float* vel, cudaStream_t s);

// Scratch of the stand-alone entry points for n points, each part 256-byte
// aligned: counters | prev | source slots | sort keys | scattered points |
// ord | rank | slots | slot contents | target records | group origins | bin
// counts | bin starts | slot-scan sums | fixed-point sums.  Non-decreasing in
// n, so its maximum over n <= m is its value at m.
__host__ __device__ constexpr size_t bs_up256(size_t b) { return (b + 255) & ~size_t(255); }
__host__ __device__ constexpr size_t bs_scratch_bytes(long long n) {
    return bs_up256(sizeof(int) * CNT_COUNT) + bs_up256(sizeof(int) * (size_t)n) +
           bs_up256(sizeof(float4) * BS_REC * (size_t)bs_slot_cap(n)) + 5 * bs_up256(sizeof(int) * (size_t)n) +
           bs_up256(sizeof(int) * (size_t)bs_slot_cap(n)) + bs_up256(sizeof(float4) * 4 * (size_t)n) +
           bs_up256(sizeof(int4) * (size_t)(bs_slot_cap(n) / BS_GROUP)) +
           bs_up256(sizeof(int) * (size_t)BS_SLOT_BLOCKS) +
           bs_up256(sizeof(long long) * 3 * (size_t)n);
}

// abi.cu
int set_error(int code, const char* msg);
int bs_standalone(const vlb_params* p, const double* pos, const int32_t* next, int32_t n, float* vel, void* scratch,
                  size_t scratch_bytes, void* stream);

// topo.cu
// Points one pass of a per-point grid covers: the top of the power-of-two
// class of the last known count n (graphs are captured again when the count
// leaves its class), at most cap.  The kernels stride over any points beyond.
inline int point_span(int n, int cap) {
    long long t = 2;
    while (t <= n) t <<= 1;
    return (int)(t < cap ? t : cap);
}
// remesh = geometry (FP64 lengths, curvature, flags; reads the points only)
// then the single-block finish, which writes the other point buffer
void launch_remesh_geometry(const VfmParams& P, Dev& d, int cur, int cap, int span, cudaStream_t s);
void launch_remesh_finish(const VfmParams& P, Dev& d, int cur, int cap, cudaStream_t s);
void launch_remesh(const VfmParams& P, Dev& d, int cur, int cap, int span, cudaStream_t s);
void launch_reconnect(const VfmParams& P, Dev& d, int cur, int cap, int span, int hsize, cudaStream_t s);
void init_hash(Dev& d, int hsize, cudaStream_t s);

}  // namespace vlb
