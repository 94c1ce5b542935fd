// C ABI of libvlb (declared in include/vlb.h): the channel runtime.  It owns
// the device buffers, sequences the kernels of one coupled step on the
// caller's stream, and moves fields between host and device.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <functional>
#include <string>
#include <vector>

#include "vlb_internal.cuh"

using namespace vlb;

// The status block on the device and in its pinned host copies: the f64
// statistics, then the int32 counters.
static constexpr size_t STATUS_BYTES = sizeof(double) * DS_COUNT + sizeof(int) * CNT_COUNT;
static constexpr size_t STATUS_SLOT = (STATUS_BYTES + 255) & ~size_t(255);  // stride of the async slots

namespace {

thread_local std::string g_last_error = "no error";

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    return fail(VLB_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace

struct vlb_channel {
    vlb_params p;
    vlb_allocator alloc;
    bool has_alloc = false;
    cudaStream_t stream = nullptr;
    Dev d;
    LbmParams lp;
    VfmParams vp;
    int cur_f = 0;     // population buffer holding the current state
    int cur_p = 0;     // point buffer holding the current filaments
    // Host record of the device state that lets a full step skip the force reset:
    bool f_clean = true;  // force grid zero everywhere (each lattice pass consumes it)
    int cap = 0;
    int hsize = 0;
    int wpp = 0;  // stream-collide warps per z plane
    int nsplit_max = 1;
    int n_hint = 0;
    long long steps = 0;
    std::vector<void*> blocks;
    size_t bytes = 0;  // device bytes allocated at create
    int* h_counters = nullptr;   // pinned
    double* h_dstats = nullptr;  // pinned
    bool timing = false;
    bool graphs = true;                      // replay captured steps when the stream allows capture
    // [steps per graph: 1 or GRAPH_MULTI][cur_f][cur_p]
    cudaGraphExec_t gexec[2][2][2] = {{{nullptr, nullptr}, {nullptr, nullptr}}, {{nullptr, nullptr}, {nullptr, nullptr}}};
    int gclass[2][2][2] = {{{-1, -1}, {-1, -1}}, {{-1, -1}, {-1, -1}}};  // filament size class at capture
    // event-timed mode: CUDA events around every launch of one kernel kind
    // (VLB_TIMED_*), in pairs, on the channel's stream
    std::vector<cudaEvent_t> ev[VLB_TIMED_KINDS];
    size_t ev_used[VLB_TIMED_KINDS] = {};
    // vlb_step_async calls in flight: each copies the status block into its
    // own pinned slot and records its own event; vlb_query completes the
    // oldest (slots q_tail .. q_head - 1, modulo VLB_ASYNC_DEPTH)
    unsigned char* h_ring = nullptr;  // pinned, VLB_ASYNC_DEPTH status blocks
    cudaEvent_t q_ev[VLB_ASYNC_DEPTH] = {};
    bool q_line[VLB_ASYNC_DEPTH] = {};  // the call stepped (its status carries the line length)
    long long q_steps[VLB_ASYNC_DEPTH] = {};  // steps queued on the channel up to the end of the call
    int q_lat[VLB_ASYNC_DEPTH] = {};          // split step: parity slot of its lattice statistics, else -1
    int done_lat = -1;
    // Split async steps (vlb_step_async of one step, overlap on): lattice pass
    // and RK stages on the channel's stream, remesh, reconnection, line length
    // and status read on the second stream, so the second-stream work of one
    // call runs beside the lattice pass of the next.  [lattice, stages,
    // topology][population parity, point parity, point parity]
    cudaGraphExec_t sgexec[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
    int sgclass[3][2] = {{-1, -1}, {-1, -1}, {-1, -1}};
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    bool b_tail = false;  // second-stream work of a split step not yet joined into the channel's stream
    int b_slot = 0;       // its slot (the slot's event follows all of that work, the status copy included)
    int last_lat = 0;     // parity slot of the last split lattice pass
    int q_head = 0, q_tail = 0;
    unsigned char done_block[STATUS_BYTES] = {};  // status block of the call vlb_query last completed
    long long done_steps = -1;                   // its step count; -1: no call completed yet
    // second stream (highest priority) and fork/join events of the multi-step graphs
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool overlap = true;  // multi-step graphs use the second stream (vlb_set_overlap)
    bool line_fresh = false;  // h_dstats[DS_LINE] holds the line length of the current points
    bool side_failed = false;  // the second stream could not be created
    double timing_ms[VLB_TIMED_KINDS] = {};
    long long timing_launches[VLB_TIMED_KINDS] = {};

    void* dalloc(size_t bytes) {
        if (bytes == 0) bytes = 16;
        bytes = (bytes + 255) & ~size_t(255);
        void* ptr = nullptr;
        if (has_alloc) {
            ptr = alloc.alloc(alloc.ctx, bytes, (void*)stream);
        } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
            ptr = nullptr;
        }
        if (ptr) {
            blocks.push_back(ptr);
            this->bytes += bytes;
        }
        return ptr;
    }
};

namespace {

void release(vlb_channel* ch) {
    cudaStreamSynchronize(ch->stream);
    if (ch->side) cudaStreamSynchronize(ch->side);
    for (void* b : ch->blocks) {
        if (ch->has_alloc) ch->alloc.free(ch->alloc.ctx, b, (void*)ch->stream);
        else cudaFree(b);
    }
    ch->blocks.clear();
    for (auto& list : ch->ev) {
        for (cudaEvent_t e : list) cudaEventDestroy(e);
        list.clear();
    }
    for (cudaEvent_t& e : ch->q_ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    for (auto& row : ch->sgexec)
        for (cudaGraphExec_t& g : row) {
            if (g) cudaGraphExecDestroy(g);
            g = nullptr;
        }
    if (ch->ev_a) cudaEventDestroy(ch->ev_a);
    if (ch->ev_b) cudaEventDestroy(ch->ev_b);
    ch->ev_a = ch->ev_b = nullptr;
    ch->b_tail = false;
    if (ch->h_ring) cudaFreeHost(ch->h_ring);
    ch->h_ring = nullptr;
    ch->q_head = ch->q_tail = 0;
    if (ch->side) cudaStreamDestroy(ch->side);
    if (ch->ev_fork) cudaEventDestroy(ch->ev_fork);
    if (ch->ev_join) cudaEventDestroy(ch->ev_join);
    ch->side = nullptr;
    ch->ev_fork = ch->ev_join = nullptr;
    for (int m = 0; m < 2; ++m)
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                if (ch->gexec[m][a][b]) {
                    cudaGraphExecDestroy(ch->gexec[m][a][b]);
                    ch->gexec[m][a][b] = nullptr;
                }
    if (ch->h_dstats) cudaFreeHost(ch->h_dstats);  // one pinned block: dstats, then counters
    ch->h_counters = nullptr;
    ch->h_dstats = nullptr;
}

int status_to_code(int st, std::string* msg) {
    if (st & ST_NAN) { *msg = "NaN/Inf in the lattice or on a filament"; return VLB_ERR_NAN; }
    if (st & ST_TOPOLOGY) { *msg = "filament successor array corrupted"; return VLB_ERR_TOPOLOGY; }
    if (st & ST_TIMEOUT) { *msg = "a device-side wait timed out"; return VLB_ERR_TIMEOUT; }
    if (st & ST_CAPACITY) { *msg = "filament point capacity (max_points) exceeded"; return VLB_ERR_CAPACITY; }
    if (st & ST_CFL) { *msg = "a filament point moved one cell or more within a step"; return VLB_ERR_CFL; }
    if (st & ST_MACH) { *msg = "Mach number |u|/c_s reached 0.05"; return VLB_ERR_MACH; }
    return VLB_OK;
}

// Make the channel's stream wait for the second-stream work of the last
// split async step, and give the status block's own mass and Mach slots the
// values of its lattice pass.  Every call that reads or changes the state
// on the channel's stream comes through here first.
void join_side(vlb_channel* ch) {
    if (!ch->b_tail) return;
    cudaStreamWaitEvent(ch->stream, ch->q_ev[ch->b_slot], 0);
    cudaMemcpyAsync(ch->d.dstats + DS_MASS, ch->d.dstats + DS_LAT + 2 * ch->last_lat, 2 * sizeof(double),
                    cudaMemcpyDeviceToDevice, ch->stream);
    ch->b_tail = false;
}

// Copy the device counters and statistics to the pinned mirrors and wait.
int sync_counters(vlb_channel* ch) {
    join_side(ch);
    cudaMemcpyAsync(ch->h_dstats, ch->d.dstats, STATUS_BYTES,
                    cudaMemcpyDeviceToHost, ch->stream);
    cudaError_t e = cudaStreamSynchronize(ch->stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    ch->n_hint = ch->h_counters[CNT_N];
    return VLB_OK;
}

void record_event(vlb_channel* ch, int kind) {
    std::vector<cudaEvent_t>& list = ch->ev[kind];
    if (ch->ev_used[kind] == list.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        list.push_back(e);
    }
    cudaEventRecord(list[ch->ev_used[kind]++], ch->stream);
}

// Flag the velocity tiles around the current points for the next lattice
// pass (the previous plane reduction cleared them).
void mark_points(vlb_channel* ch) {
    launch_mark_umask(ch->lp.g, ch->d.pos[ch->cur_p], ch->d.counters, ch->cap, ch->d.umask, ch->stream);
}

// The lattice pass: stream-collide and plane reduction (tiles already
// flagged, or every tile with all_u).
// stats != nullptr: the plane reduction writes the mass and max Mach there
// (as [0], [1]) instead of into the status block's own slots.
void lattice_pass(vlb_channel* ch, bool all_u = false, double* stats = nullptr) {
    Dev& d = ch->d;
    if (ch->timing) record_event(ch, VLB_TIMED_LBM);
    LbmParams L = ch->lp;
    L.all_u = all_u ? 1 : 0;
    launch_lbm_step(L, d.f[ch->cur_f], d.f[ch->cur_f ^ 1], d.F, d.U, d.fmask, d.umask, d.part, ch->stream);
    if (ch->timing) record_event(ch, VLB_TIMED_LBM);
    ch->cur_f ^= 1;
    // the pass consumed the force grid: the plane reduction resets it and clears both tile flags
    LbmParams R = ch->lp;
    if (stats) R.dstats = stats - DS_MASS;
    launch_plane_vs(R, d.part, d.F, d.umask, d.fmask, ch->stream);
    ch->f_clean = true;
}

void phase_lbm(vlb_channel* ch) {
    mark_points(ch);
    lattice_pass(ch);
}

// Whether the Biot-Savart kernel applies the equation of motion itself: by
// default from BS_ACC_MAX points on, where it sums partial sums per target
// tile (below, the fixed-point accumulator and a separate kernel are faster);
// VLB_FUSED_EOM=1 / 0 in the environment forces it on / off.
bool fused_eom(int n) {
    const char* v = getenv("VLB_FUSED_EOM");
    return v ? v[0] != '0' : n >= BS_ACC_MAX;
}

// Stage-0 geometry and Biot-Savart sum of the first sub-step: they read only
// the points, so they may run before the lattice pass is done.
// Order of the Biot-Savart sources for the current filament size: spatial
// from BS_SORT_MIN points on (the pair sums are compute-bound there and
// compact groups of sources take the cheap pair path), point order below.
BsOrder bs_order(vlb_channel* ch) {
    BsOrder o;
    o.sorted = ch->n_hint >= BS_SORT_MIN ? 1 : 0;
    o.ord = ch->d.bs_ord;
    o.rank = ch->d.bs_rank;
    o.slot = ch->d.bs_slot;
    o.pt = ch->d.bs_pt;
    o.org = ch->d.bs_org;
    o.tgt = ch->d.bs_tgt;
    return o;
}

// The spatial order (in point order below BS_SORT_MIN points) and the source
// slots of the current points, before the first stage geometry of a step;
// they then serve every RK stage of the step.
void bs_sort(vlb_channel* ch, const BsOrder& o, cudaStream_t s) {
    Dev& d = ch->d;
    const int span = point_span(ch->n_hint, ch->cap);
    if (o.sorted)
        launch_bs_sort(ch->vp.g, d.pos[ch->cur_p], ch->cap, d.counters, d.bs_key, d.bs_hist, d.bs_ord, d.bs_rank, s);
    launch_bs_slots(d.pos[ch->cur_p], d.next[ch->cur_p], ch->cap, span, d.counters, o, d.bs_bsum, s);
}

void vfm_pre(vlb_channel* ch, cudaStream_t s) {
    Dev& d = ch->d;
    const VfmParams& V = ch->vp;
    const int* prev = d.prev[ch->cur_p];
    const BsOrder o = bs_order(ch);
    bs_sort(ch, o, s);
    launch_geometry_stage(V, d.pos[ch->cur_p], d.next[ch->cur_p], prev, d.counters, ch->cap,
                          point_span(ch->n_hint, ch->cap), d.geo, d.seg, d.s0, o, s);
    launch_biot_savart(V.g, V.kappa, d.seg, prev, d.counters, d.tile_ticket, ch->cap, ch->n_hint, d.bsp, d.vbs, s, o,
                       nullptr, V.nfaces, V.face_code, d.geo, d.vacc);
}

// Arguments of one filament step on the current points, v_n and V_s.
EomArgs eom_args(vlb_channel* ch) {
    Dev& d = ch->d;
    EomArgs ea = {};
    ea.P = ch->vp;
    ea.cap = ch->cap;
    ea.s0 = d.s0;
    ea.st = d.st;
    ea.pos_out = d.pos[ch->cur_p];
    ea.acc = d.acc;
    ea.vel1 = d.vel1;
    ea.geo = d.geo;
    ea.U = d.U;
    ea.Vs = d.Vs;
    ea.F = d.F;
    ea.fmask = d.fmask;
    ea.counters = d.counters;
    return ea;
}

// One filament step: the RK4 stages of every sub-step (Eqs. 3-4, 10-11) on
// the current points; the first stage's geometry and Biot-Savart sum are
// skipped when vfm_pre queued them.
void vfm_step(vlb_channel* ch, bool pre_done, cudaStream_t s) {
    Dev& d = ch->d;
    const VfmParams& V = ch->vp;
    const int* next = d.next[ch->cur_p];
    const int* prev = d.prev[ch->cur_p];
    const int nsub = ch->p.vfm_substeps > 0 ? ch->p.vfm_substeps : 1;
    EomArgs ea = eom_args(ch);
    const BsOrder o = bs_order(ch);
    for (int sub = 0; sub < nsub; ++sub) {
        const int spread = (sub == 0 && ch->p.couple) ? 1 : 0;
        if (spread && !ch->f_clean) launch_zero_force(ch->lp.g, d.F, d.fmask, s);
        if (spread) ch->f_clean = false;
        for (int stage = 0; stage < 4; ++stage) {
            ea.stage = stage;
            ea.spread = spread;
            ea.first = sub == 0 ? 1 : 0;
            // below the fused size the Biot-Savart sums arrive in d.vacc
            long long* vacc = bs_uses_vacc(ch->n_hint) ? d.vacc : nullptr;
            if (pre_done && sub == 0 && stage == 0) {
                launch_eom(ea, d.vbs, s, vacc);
                continue;
            }
            if (sub == 0 && stage == 0) bs_sort(ch, o, s);
            launch_geometry_stage(V, stage == 0 ? ea.pos_out : d.st, next, prev, d.counters, ch->cap,
                                  point_span(ch->n_hint, ch->cap), d.geo, d.seg, stage == 0 ? d.s0 : nullptr, o, s);
            const bool timed = ch->timing && s == ch->stream;
            if (timed) record_event(ch, VLB_TIMED_BIOT_SAVART);
            if (fused_eom(ch->n_hint)) {
                launch_biot_savart(V.g, V.kappa, d.seg, prev, d.counters, d.tile_ticket, ch->cap, ch->n_hint, d.bsp,
                                   d.vbs, s, o, &ea, V.nfaces, V.face_code, d.geo);
                if (timed) record_event(ch, VLB_TIMED_BIOT_SAVART);
            } else {
                launch_biot_savart(V.g, V.kappa, d.seg, prev, d.counters, d.tile_ticket, ch->cap, ch->n_hint, d.bsp,
                                   d.vbs, s, o, nullptr, V.nfaces, V.face_code, d.geo, vacc);
                if (timed) record_event(ch, VLB_TIMED_BIOT_SAVART);
                launch_eom(ea, d.vbs, s, vacc);
            }
        }
    }
}

void phase_vfm(vlb_channel* ch) { vfm_step(ch, false, ch->stream); }

void run_phases_body(vlb_channel* ch, int mask) {
    if (mask & VLB_PHASE_LBM) phase_lbm(ch);
    if (mask & VLB_PHASE_VFM) phase_vfm(ch);
    if (mask & VLB_PHASE_REMESH) {
        launch_remesh(ch->vp, ch->d, ch->cur_p, ch->cap, point_span(ch->n_hint, ch->cap), ch->stream);
        ch->cur_p ^= 1;
    }
    if (mask & VLB_PHASE_RECONNECT) {
        launch_reconnect(ch->vp, ch->d, ch->cur_p, ch->cap, point_span(ch->n_hint, ch->cap), ch->hsize, ch->stream);
        ch->cur_p ^= 1;
    }
}

void run_phases(vlb_channel* ch, int mask) {
    const bool was = tl_no_pdl;
    if (ch->timing) tl_no_pdl = true;
    run_phases_body(ch, mask);
    tl_no_pdl = was;
}
int finish(vlb_channel* ch) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    int rc = sync_counters(ch);
    if (rc) return rc;
    std::string msg;
    rc = status_to_code(ch->h_counters[CNT_STATUS], &msg);
    if (rc) return fail(rc, msg);
    return VLB_OK;
}

bool valid_axis_params(const vlb_params* p, std::string* why) {
    for (int a = 0; a < 3; ++a) {
        if (p->n[a] < 1) { *why = "n must be >= 1 on every axis"; return false; }
        if (p->wall[a] != 0 && p->wall[a] != 1) { *why = "wall must be 0 or 1"; return false; }
    }
    if (p->stream_axis != 2) { *why = "stream_axis must be 2 (z) in this library"; return false; }
    if (p->wall_images != 0 && p->wall_images != 1) { *why = "wall_images must be 0 or 1"; return false; }
    if (!(p->tau > 0.5)) { *why = "tau must exceed 1/2"; return false; }
    if (!(p->rho0 > 0.0)) { *why = "rho0 must be positive"; return false; }
    if (!(p->dxi_min > 0.0) || !(p->dxi_max > p->dxi_min) || !(p->dxi_max < 1.0)) {
        *why = "need 0 < dxi_min < dxi_max < 1";
        return false;
    }
    if (!(p->rho_s_over_rho_n > 0.0) || !(p->core_a > 0.0) || !(p->kappa >= 0.0)) {
        *why = "rho_s_over_rho_n, core_a must be positive and kappa >= 0";
        return false;
    }
    if (p->max_points < 0 || p->vfm_substeps < 1) {
        *why = "max_points >= 0 and vfm_substeps >= 1 required";
        return false;
    }
    if (p->storage != VLB_STORE_F32 && p->storage != VLB_STORE_F16 && p->storage != VLB_STORE_BF16) {
        *why = "storage must be VLB_STORE_F32, VLB_STORE_F16 or VLB_STORE_BF16";
        return false;
    }
    if (p->force_form != 0 && p->force_form != 1) { *why = "force_form must be 0 or 1"; return false; }
    if (p->heater_vn != 0.0 && !p->wall[2]) { *why = "heater_vn needs walls on z"; return false; }
    if (p->pin_vn != 0.0 && p->wall[2]) { *why = "pin_vn needs a periodic z axis"; return false; }
    const double u0 = sqrt(p->init_vn[0] * p->init_vn[0] + p->init_vn[1] * p->init_vn[1] + p->init_vn[2] * p->init_vn[2]);
    if (!(sqrt(3.0) * u0 < 0.05) || !(sqrt(3.0) * fabs(p->heater_vn) < 0.05) || !(sqrt(3.0) * fabs(p->pin_vn) < 0.05)) {
        *why = "imposed velocities exceed Mach 0.05";
        return false;
    }
    const long long cells = (long long)p->n[0] * p->n[1] * p->n[2];
    if (cells > (1LL << 31) / 19) { *why = "lattice too large"; return false; }
    return true;
}

}  // namespace

namespace vlb {

int set_error(int code, const char* msg) { return fail(code, msg); }

thread_local bool tl_no_pdl = false;

bool pdl_enabled() {
    static const bool on = [] {
        const char* v = getenv("VLB_PDL");
        return !(v && v[0] == '0');
    }();
    return on;
}

// Stand-alone Biot-Savart velocity on caller-provided device buffers; the
// scratch layout is the one bs_scratch_bytes sizes, each part 256-byte
// aligned.  The split sums are added in fixed point (exact, in any order) and
// converted to float at the end.  Allocates nothing.
int bs_standalone(const vlb_params* p, const double* pos, const int32_t* next, int32_t n, float* vel, void* scratch,
                  size_t scratch_bytes, void* stream) {
    if (!p || n < 0 || (n > 0 && (!pos || !next || !vel || !scratch)))
        return fail(VLB_ERR_INVALID_ARG, "bad Biot-Savart arguments");
    if (n == 0) return VLB_OK;
    for (int a = 0; a < 3; ++a)
        if (p->n[a] < 1 || (p->wall[a] != 0 && p->wall[a] != 1)) return fail(VLB_ERR_INVALID_ARG, "bad box");
    if (scratch_bytes < bs_scratch_bytes(n)) return fail(VLB_ERR_INVALID_ARG, "scratch too small");
    if (((uintptr_t)scratch & 255u) != 0) return fail(VLB_ERR_INVALID_ARG, "scratch must be 256-byte aligned");
    Grid g;
    g.nx = p->n[0];
    g.ny = p->n[1];
    g.nz = p->n[2];
    for (int a = 0; a < 3; ++a) g.wall[a] = p->wall[a];
    g.ncell = (long long)g.nx * g.ny * g.nz;
    g.tnx = g.tny = g.tnz = 1;
    const size_t slots = (size_t)bs_slot_cap(n);
    char* base = (char*)scratch;
    auto take = [&](size_t bytes) {
        char* q = base;
        base += bs_up256(bytes);
        return (void*)q;
    };
    int* counters = (int*)take(sizeof(int) * CNT_COUNT);
    int* prev = (int*)take(sizeof(int) * (size_t)n);
    float4* seg = (float4*)take(sizeof(float4) * BS_REC * slots);
    int* key = (int*)take(sizeof(int) * (size_t)n);
    int* hist = (int*)take(sizeof(int) * (size_t)n);
    int* ord = (int*)take(sizeof(int) * (size_t)n);
    int* rank = (int*)take(sizeof(int) * (size_t)n);
    int* slot = (int*)take(sizeof(int) * (size_t)n);
    int* pt = (int*)take(sizeof(int) * slots);
    float4* tgt = (float4*)take(sizeof(float4) * 4 * (size_t)n);
    int4* org = (int4*)take(sizeof(int4) * (slots / BS_GROUP));
    int* bsum = (int*)take(sizeof(int) * BS_SLOT_BLOCKS);
    long long* vacc = (long long*)take(sizeof(long long) * 3 * (size_t)n);
    cudaStream_t s = (cudaStream_t)stream;
    BsOrder o;
    o.sorted = n >= BS_SORT_MIN ? 1 : 0;
    o.ord = ord;
    o.rank = rank;
    o.slot = slot;
    o.pt = pt;
    o.org = org;
    o.tgt = tgt;
    cudaMemsetAsync(vacc, 0, sizeof(long long) * 3 * (size_t)n, s);
    launch_bs_standalone_prep(g, pos, next, n, prev, seg, counters, o, key, hist, bsum, s);
    launch_biot_savart(g, p->kappa, seg, prev, counters, nullptr, n, n, nullptr, vel, s, o, nullptr, 0, nullptr,
                       nullptr, vacc);
    launch_bs_unfix(vacc, n, vel, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "Biot-Savart launch");
    return VLB_OK;
}

}  // namespace vlb

extern "C" {

const char* vlb_last_error(void) { return g_last_error.c_str(); }

size_t vlb_channel_bytes(const vlb_params* p) {
    std::string why;
    if (!p || !valid_axis_params(p, &why)) return 0;
    auto up = [](size_t b) { return ((b ? b : 16) + 255) & ~size_t(255); };
    const size_t C = (size_t)p->n[0] * p->n[1] * p->n[2];
    const size_t cap = p->max_points > 0 ? (size_t)p->max_points : 1;
    const size_t nt = (size_t)((p->n[0] + 7) >> 3) * ((p->n[1] + 7) >> 3) * ((p->n[2] + 7) >> 3);
    size_t h = 1;
    while (h < 2 * cap) h <<= 1;
    const size_t esize = p->storage == VLB_STORE_F32 ? 4 : 2;
    const size_t wpp = (size_t)((p->n[0] * p->n[1] + 255) / 256) * 8;  // warps per plane, any block shape
    size_t b = 2 * up(esize * 19 * C) + up(8 * 3 * C) + up(4 * 3 * C) + 2 * up(nt) + up(4 * 3 * wpp * p->n[2]);
    b += 3 * up(8 * (size_t)p->n[2]) + up(4 * (size_t)p->n[2]) + up(8 * DS_COUNT) + up(4 * CNT_COUNT);
    size_t nfaces = 0;
    if (p->wall_images)
        for (int a = 0; a < 3; ++a) nfaces += p->wall[a] ? 2 : 0;
    const size_t capg = (size_t)bs_slot_cap((long long)cap);
    b += 2 * (up(24 * cap) + 2 * up(4 * cap)) + 6 * up(24 * cap) + up(8 * cap) + up(32 * cap) +
         up(sizeof(float4) * BS_REC * capg * (1 + nfaces));
    b += up(12 * cap * (size_t)bs_max_splits((int)cap, sm_count())) + up(12 * cap) + up(24 * cap) +
         up(4 * ((cap + 127) / 128));
    b += 5 * up(4 * cap) + up(16 * (capg / BS_GROUP)) +
         up(4 * BS_SLOT_BLOCKS) + up(4 * capg) + up(64 * cap);
    b += 2 * up(cap) + 4 * up(4 * cap) + up(4 * h) + 2 * up(4 * cap) + up(16 * cap) + up(8 * cap);
    const size_t nc = cap / 2 + 1;
    b += 4 * up(4 * nc) + up(8 * nc) + up(4 * cap) + up(8 * ((cap + 255) / 256));
    return b;
}

int vlb_create_channel(const vlb_params* p, const vlb_allocator* alloc, void* stream, vlb_channel** out) {
    if (!p || !out) return fail(VLB_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    std::string why;
    if (!valid_axis_params(p, &why)) return fail(VLB_ERR_INVALID_ARG, why);
    if (alloc && (!alloc->alloc || !alloc->free)) return fail(VLB_ERR_INVALID_ARG, "allocator without callbacks");
    vlb_channel* ch = new vlb_channel();
    ch->p = *p;
    if (alloc) {
        ch->alloc = *alloc;
        ch->has_alloc = true;
    }
    ch->stream = (cudaStream_t)stream;
    Grid g;
    g.nx = p->n[0];
    g.ny = p->n[1];
    g.nz = p->n[2];
    for (int a = 0; a < 3; ++a) g.wall[a] = p->wall[a];
    g.ncell = (long long)g.nx * g.ny * g.nz;
    g.tnx = (g.nx + 7) >> TILE_SHIFT;
    g.tny = (g.ny + 7) >> TILE_SHIFT;
    g.tnz = (g.nz + 7) >> TILE_SHIFT;
    LbmParams& L = ch->lp;
    L.g = g;
    L.omega = (float)(1.0 / p->tau);
    L.pref = (float)(1.0 - 1.0 / (2.0 * p->tau));
    L.rho0 = (float)p->rho0;
    for (int a = 0; a < 3; ++a) L.body[a] = (float)p->body_force[a];
    L.body_on = (p->body_force[0] != 0.0 || p->body_force[1] != 0.0 || p->body_force[2] != 0.0) ? 1 : 0;
    L.heater = (float)p->heater_vn;
    L.pin = (float)p->pin_vn;
    L.pin_on = p->pin_vn != 0.0 ? 1 : 0;
    {
        // Launch shape of the stream-collide kernel, chosen from measurements on
        // GB300 (lattices of 32^3 to 128x128x1024): with FP32 storage one cell
        // per thread in 128-thread blocks was fastest everywhere; with 16-bit
        // storage two cells per thread (packed loads, stores and arithmetic),
        // when nx is even.  VLB_LBM_VEC (1, 2, 4; 16-bit storage: 1, 2) and
        // VLB_LBM_BLOCK (128, 256) override it.
        const bool half = p->storage != VLB_STORE_F32;
        int vec = half && g.nx % 2 == 0 ? 2 : 1;
        if (const char* e = getenv("VLB_LBM_VEC")) {
            const int v = atoi(e);
            if ((v == 1 || v == 2 || (v == 4 && !half)) && g.nx % v == 0) vec = v;
        }
        int blk = 128;
        if (const char* e = getenv("VLB_LBM_BLOCK")) {
            const int b = atoi(e);
            if (b == 128 || b == 256) blk = b;
        }
        L.vec = vec;
        // exact division by nx through a multiply-high (Granlund-Montgomery),
        // checked here for every in-plane index the kernel can form
        {
            const unsigned d = (unsigned)g.nx;
            int sh = 0;
            while ((1ull << sh) < d) ++sh;
            const int shift = 32 + sh;
            const unsigned long long m = ((1ull << shift) + d - 1) / d;
            bool exact = true;
            const unsigned lim = (unsigned)g.nx * (unsigned)g.ny;
            for (unsigned xy = 0; xy < lim && exact; ++xy) exact = ((xy * m) >> shift) == xy / d;
            if (!exact) {
                delete ch;
                return fail(VLB_ERR_INVALID_ARG, "no exact multiply-high division for this nx");
            }
            L.nx_magic = m;
            L.nx_shift = shift;
        }
        L.block = blk;
        L.storage = p->storage;
        // Evict-first hints on the population traffic when one population
        // buffer fits in L2: the filament data then stays in L2 beside the
        // streaming lattice (measured on 64x64x256: step 0.1287 -> 0.1216 ms).
        // Larger lattices gain nothing from L2 and the hints cost the pass up to
        // 8% there.  VLB_LBM_STREAM_HINT (0, 1) overrides.
        int l2 = 0;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
        const double pop_bytes = (p->storage == VLB_STORE_F32 ? 4.0 : 2.0) * 19.0 * (double)g.ncell;
        L.stream_hint = pop_bytes <= (double)l2 ? 1 : 0;
        if (const char* e = getenv("VLB_LBM_STREAM_HINT")) L.stream_hint = e[0] == '1' ? 1 : 0;
    }
    {
        // float shift constants s_i = fl(fl(w_i) rho0) as the kernels form them
        const double wexact[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};
        const float wf[3] = {1.f / 3.f, 1.f / 18.f, 1.f / 36.f};
        const int mult[3] = {1, 6, 12};
        double ssum = 0.0;
        for (int k = 0; k < 3; ++k) {
            const float sk = wf[k] * (float)p->rho0;
            ssum += mult[k] * (double)sk;
            L.dw[k] = (float)(wexact[k] * p->rho0 - (double)sk);
        }
        L.dr0 = (float)(ssum - p->rho0);
    }
    VfmParams& V = ch->vp;
    V.g = g;
    V.kappa = p->kappa;
    V.alpha = p->alpha;
    V.alpha_p = p->alpha_p;
    V.ratio = p->rho_s_over_rho_n;
    V.rho0 = p->rho0;
    V.core_a = p->core_a;
    V.dmin = p->dxi_min;
    V.dmax = p->dxi_max;
    V.dt = 1.0 / (double)p->vfm_substeps;
    V.couple = p->couple;
    V.force_form = p->force_form;
    V.kq_f = (float)(p->kappa / (4.0 * 3.14159265358979323846));
    V.beta_c_f = (float)log(2.0 / (exp(0.25) * p->core_a));
    V.alpha_f = (float)p->alpha;
    V.alpha_p_f = (float)p->alpha_p;
    V.gscale_f = (float)(-p->rho_s_over_rho_n * p->rho0 * p->kappa);
    V.nfaces = 0;
    if (p->wall_images)
        for (int a = 0; a < 3; ++a)
            if (p->wall[a])
                for (int side = 0; side < 2; ++side) V.face_code[V.nfaces++] = 2 * a + side;

    const long long C = g.ncell;
    const int cap = p->max_points > 0 ? p->max_points : 1;
    ch->cap = cap;
    int h = 1;
    while (h < 2 * cap) h <<= 1;
    ch->hsize = h;
    ch->wpp = lbm_warps_per_plane(L);
    const int nsm = bs_max_splits(cap, sm_count());
    ch->nsplit_max = nsm;
    const size_t capg = (size_t)bs_slot_cap(cap);  // source slots: a point and a gap slot each, whole groups
    const int ntiles = g.tnx * g.tny * g.tnz;
    Dev& d = ch->d;
    bool ok = true;
    auto A = [&](size_t bytes) {
        void* q = ch->dalloc(bytes);
        if (!q) ok = false;
        return q;
    };
    const size_t esize = p->storage == VLB_STORE_F32 ? 4 : 2;
    d.f[0] = A(esize * 19 * (size_t)C);
    d.f[1] = A(esize * 19 * (size_t)C);
    d.F = (long long*)A(sizeof(long long) * 3 * (size_t)C);
    d.U = (float*)A(sizeof(float) * 3 * (size_t)C);
    d.Vs = (double*)A(sizeof(double) * (size_t)g.nz);
    d.fmask = (uint8_t*)A((size_t)ntiles);
    d.umask = (uint8_t*)A((size_t)ntiles);
    d.part = (float*)A(sizeof(float) * 3 * (size_t)ch->wpp * g.nz);
    d.plane = (double*)A(sizeof(double) * 3 * (size_t)g.nz);
    d.plane_ticket = (int*)A(sizeof(int) * (size_t)g.nz);
    // statistics and counters in one block, read back with one copy
    d.dstats = (double*)A(STATUS_BYTES);
    d.counters = d.dstats ? (int*)(d.dstats + DS_COUNT) : nullptr;
    const size_t P3 = sizeof(double) * 3 * (size_t)cap;
    for (int b = 0; b < 2; ++b) {
        d.pos[b] = (double*)A(P3);
        d.next[b] = (int*)A(sizeof(int) * (size_t)cap);
        d.prev[b] = (int*)A(sizeof(int) * (size_t)cap);
    }
    d.s0 = (double*)A(P3);
    d.st = (double*)A(P3);
    d.acc = (double*)A(P3);
    d.vel1 = (double*)A(P3);
    d.spp = (double*)A(P3);
    d.seglen = (double*)A(sizeof(double) * (size_t)cap);
    d.geo = (float4*)A(sizeof(float4) * 2 * (size_t)cap);
    d.seg = (float4*)A(sizeof(float4) * BS_REC * capg * (size_t)(1 + V.nfaces));  // segments, then wall images
    d.bs_key = (int*)A(sizeof(int) * (size_t)cap);
    d.bs_hist = (int*)A(sizeof(int) * (size_t)cap);
    d.bs_ord = (int*)A(sizeof(int) * (size_t)cap);
    d.bs_rank = (int*)A(sizeof(int) * (size_t)cap);
    d.bs_org = (int4*)A(sizeof(int4) * (capg / BS_GROUP));
    d.bs_slot = (int*)A(sizeof(int) * (size_t)cap);
    d.bs_pt = (int*)A(sizeof(int) * capg);
    d.bs_tgt = (float4*)A(sizeof(float4) * 4 * (size_t)cap);
    d.bs_bsum = (int*)A(sizeof(int) * BS_SLOT_BLOCKS);
    d.bsp = (float*)A(sizeof(float) * 3 * (size_t)cap * (size_t)nsm);
    d.vbs = (float*)A(sizeof(float) * 3 * (size_t)cap);
    d.vacc = (long long*)A(sizeof(long long) * 3 * (size_t)cap);
    d.tile_ticket = (int*)A(sizeof(int) * (size_t)((cap + BS_TPB - 1) / BS_TPB));
    d.flags = (uint8_t*)A((size_t)cap);
    d.alive = (uint8_t*)A((size_t)cap);
    d.nnext = (int*)A(sizeof(int) * (size_t)cap);
    d.newidx = (int*)A(sizeof(int) * (size_t)cap);
    d.hkey = (int*)A(sizeof(int) * (size_t)cap);
    d.hhead = (int*)A(sizeof(int) * (size_t)h);
    d.hlink = (int*)A(sizeof(int) * (size_t)cap);
    d.hpos = (float4*)A(sizeof(float4) * (size_t)cap);
    d.nn = (int*)A(sizeof(int) * (size_t)cap);
    d.nd2 = (double*)A(sizeof(double) * (size_t)cap);
    const size_t nc = (size_t)cap / 2 + 1;
    d.cand_i = (int*)A(sizeof(int) * nc);
    d.cand_a = (int*)A(sizeof(int) * nc);
    d.cand_b = (int*)A(sizeof(int) * nc);
    d.cand_d2 = (double*)A(sizeof(double) * nc);
    d.cand_order = (int*)A(sizeof(int) * nc);
    d.stamp = (int*)A(sizeof(int) * (size_t)cap);
    d.line_part = (double*)A(sizeof(double) * (size_t)((cap + 255) / 256));
    if (!ok) {
        release(ch);
        delete ch;
        return fail(VLB_ERR_OOM, "device allocation failed");
    }
    if (cudaMallocHost((void**)&ch->h_dstats, STATUS_BYTES) == cudaSuccess)
        ch->h_counters = (int*)(ch->h_dstats + DS_COUNT);
    if (!ch->h_dstats) {
        release(ch);
        delete ch;
        return fail(VLB_ERR_OOM, "pinned host allocation failed");
    }
    cudaStream_t s = ch->stream;
    cudaMemsetAsync(d.F, 0, sizeof(long long) * 3 * (size_t)C, s);
    cudaMemsetAsync(d.fmask, 0, (size_t)ntiles, s);
    cudaMemsetAsync(d.umask, 0, (size_t)ntiles, s);
    cudaMemsetAsync(d.counters, 0, sizeof(int) * CNT_COUNT, s);
    cudaMemsetAsync(d.plane_ticket, 0, sizeof(int) * (size_t)g.nz, s);
    L.plane_ticket = d.plane_ticket;
    L.plane = d.plane;
    L.Vs = d.Vs;
    L.dstats = d.dstats;
    L.counters = d.counters;
    L.inv_ratio = 1.0 / p->rho_s_over_rho_n;
    cudaMemsetAsync(d.dstats, 0, sizeof(double) * DS_COUNT, s);
    cudaMemsetAsync(d.stamp, 0, sizeof(int) * (size_t)cap, s);
    cudaMemsetAsync(d.vacc, 0, sizeof(long long) * 3 * (size_t)cap, s);
    // the stage-1 velocity export starts at zero, as in the oracle (rows past
    // the current count keep what an earlier, larger advance left)
    cudaMemsetAsync(d.vel1, 0, sizeof(double) * 3 * (size_t)cap, s);
    cudaMemsetAsync(d.bsp, 0, sizeof(float) * 3 * (size_t)cap * (size_t)nsm, s);
    cudaMemsetAsync(d.tile_ticket, 0, sizeof(int) * (size_t)((cap + BS_TPB - 1) / BS_TPB), s);
    init_hash(d, h, s);
    launch_lbm_init(L, d.f[0], d.U, p->init_vn, s);
    std::vector<double> vs((size_t)g.nz, -(1.0 / p->rho_s_over_rho_n) * p->init_vn[2]);
    double mass = p->rho0 * (double)C;
    cudaMemcpyAsync(d.Vs, vs.data(), sizeof(double) * vs.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d.dstats + DS_MASS, &mass, sizeof(double), cudaMemcpyHostToDevice, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "channel initialisation");
        release(ch);
        delete ch;
        return rc;
    }
    *out = ch;
    return VLB_OK;
}

void vlb_destroy(vlb_channel* ch) {
    if (!ch) return;
    release(ch);
    delete ch;
}

int vlb_seed_vortices(vlb_channel* ch, const double* xyz, const int32_t* next, int32_t n) {
    if (!ch || n < 0 || (n > 0 && (!xyz || !next))) return fail(VLB_ERR_INVALID_ARG, "bad seed arguments");
    join_side(ch);
    ch->line_fresh = false;
    if (n > ch->cap || (n > 0 && ch->p.max_points == 0)) return fail(VLB_ERR_CAPACITY, "more points than max_points");
    std::vector<char> seen((size_t)n, 0);
    std::vector<double> soa(3 * (size_t)ch->cap, 0.0);
    std::vector<int> prv((size_t)(n > 0 ? n : 1), -1);
    for (int i = 0; i < n; ++i) {
        const int q = next[i];
        if (q < -1 || q >= n || (q >= 0 && seen[(size_t)q]))
            return fail(VLB_ERR_TOPOLOGY, "next[] must describe closed loops and open lines");
        if (q >= 0) {
            seen[(size_t)q] = 1;
            prv[(size_t)q] = i;
        }
        for (int a = 0; a < 3; ++a) {
            double v = xyz[3 * (size_t)i + a];
            if (v != v || isinf(v)) return fail(VLB_ERR_INVALID_ARG, "non-finite position");
            const double L = (double)ch->p.n[a];
            if (ch->p.wall[a]) {
                if (v <= -0.5 || v >= L - 0.5) return fail(VLB_ERR_INVALID_ARG, "point outside the walls");
                const double lo = -0.5 + 0.5 * ch->p.dxi_min, hi = L - 0.5 - 0.5 * ch->p.dxi_min;
                if (v < lo) v = lo;
                if (v > hi) v = hi;
            } else {
                if (v < 0.0) v += L;
                else if (v >= L) v -= L;
                if (v < 0.0 || v >= L) return fail(VLB_ERR_INVALID_ARG, "periodic coordinate more than one box away");
            }
            soa[(size_t)a * ch->cap + i] = v;
        }
    }
    // Open ends go onto the nearest wall clamp bound within dxi_max (order x-,
    // x+, y-, y+, z-, z+ on ties).
    for (int i = 0; i < n; ++i) {
        if (next[i] < 0 && prv[(size_t)i] < 0) return fail(VLB_ERR_TOPOLOGY, "isolated point");
        if (next[i] >= 0 && prv[(size_t)i] >= 0) continue;
        int best_a = -1;
        double best_d = 0.0, best_b = 0.0;
        for (int a = 0; a < 3; ++a) {
            if (!ch->p.wall[a]) continue;
            const double lo = -0.5 + 0.5 * ch->p.dxi_min, hi = (double)ch->p.n[a] - 0.5 - 0.5 * ch->p.dxi_min;
            const double x = soa[(size_t)a * ch->cap + i];
            const double dl = x - lo, dh = hi - x;
            if (best_a < 0 || dl < best_d) { best_a = a; best_d = dl; best_b = lo; }
            if (dh < best_d) { best_a = a; best_d = dh; best_b = hi; }
        }
        if (best_a < 0 || best_d > ch->p.dxi_max)
            return fail(VLB_ERR_TOPOLOGY, "open end farther than dxi_max from every wall");
        soa[(size_t)best_a * ch->cap + i] = best_b;
    }
    Dev& d = ch->d;
    cudaStream_t s = ch->stream;
    const int b = ch->cur_p;
    cudaMemcpyAsync(d.pos[b], soa.data(), sizeof(double) * 3 * (size_t)ch->cap, cudaMemcpyHostToDevice, s);
    if (n > 0) {
        cudaMemcpyAsync(d.next[b], next, sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d.prev[b], prv.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, s);
    }
    cudaMemcpyAsync(d.counters + CNT_N, &n, sizeof(int), cudaMemcpyHostToDevice, s);
    const int dirty = 1;  // the seeded loops and lines are checked for size by the next remesh
    cudaMemcpyAsync(d.counters + CNT_DIRTY, &dirty, sizeof(int), cudaMemcpyHostToDevice, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "seed copy");
    ch->n_hint = n;
    return VLB_OK;
}

// One coupled step, replayed from a CUDA graph captured on first use for the
// current buffer parities (the population buffers alternate every step; the
// point buffers flip twice per step).  Capture needs a real stream, so the
// legacy default stream and the timing mode launch the kernels directly.
namespace {
int size_class(int n) {
    int c = 0;
    while (n > 1) {
        n >>= 1;
        ++c;
    }
    return c;
}

// The second stream (highest priority) and the fork/join events of the
// overlapped graphs, created when first needed.  False if they cannot be made:
// the graphs then keep their steps in sequence.
bool ensure_side(vlb_channel* ch) {
    if (ch->side) return true;
    if (ch->side_failed) return false;
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&ch->side, cudaStreamNonBlocking, hi) != cudaSuccess ||
        (!ch->ev_fork && cudaEventCreateWithFlags(&ch->ev_fork, cudaEventDisableTiming) != cudaSuccess) ||
        (!ch->ev_join && cudaEventCreateWithFlags(&ch->ev_join, cudaEventDisableTiming) != cudaSuccess)) {
        cudaGetLastError();
        if (ch->side) cudaStreamDestroy(ch->side);
        ch->side = nullptr;
        ch->side_failed = true;
        return false;
    }
    return true;
}

// Steps per multi-step graph (even, so both buffer parities are restored).
constexpr int GRAPH_MULTI = 8;

// nst full steps for a multi-step graph, on two streams.  The lattice pass
// of step s + 1 reads and writes nothing that the remesh and reconnection of
// step s touch (populations, force and velocity grids against the point
// arrays and topology scratch; counters and stats in separate slots or by
// atomics), nor what the stage-0 geometry and Biot-Savart sum of step s + 1
// read (the points only).  So that filament chain runs on the second stream
// alongside the lattice pass, forked and joined inside the graph.  The chain
// is a row of small, latency-bound launches; its stream has the highest
// priority, so its blocks go ahead of waiting stream-collide blocks.  (Run
// alongside the RK stages instead, the lattice pass slowed the Biot-Savart
// launches more than it gained.)  The points of a lattice pass are not known
// when it starts, so it writes v_n in every tile instead of the tiles around
// the points: the same values where the filaments read them.  The result is
// the same, bit for bit, as in sequence.
void run_steps_forked(vlb_channel* ch, int nst) {
    Dev& d = ch->d;
    const bool pre = !fused_eom(ch->n_hint);
    phase_lbm(ch);  // pass 0, tiles flagged around the points
    cudaEventRecord(ch->ev_fork, ch->stream);
    cudaStreamWaitEvent(ch->side, ch->ev_fork, 0);
    for (int s = 0; s < nst; ++s) {
        vfm_step(ch, s > 0 && pre, ch->side);
        // The remesh geometry runs before the fork: alone it takes about half
        // of what it takes beside the stream-collide pass, and the lattice
        // branch is the shorter one by about as much.
        launch_remesh_geometry(ch->vp, d, ch->cur_p, ch->cap, point_span(ch->n_hint, ch->cap), ch->side);
        if (s + 1 < nst) {
            cudaEventRecord(ch->ev_fork, ch->side);
            cudaStreamWaitEvent(ch->stream, ch->ev_fork, 0);
            lattice_pass(ch, true);
            cudaEventRecord(ch->ev_join, ch->stream);
        }
        launch_remesh_finish(ch->vp, d, ch->cur_p, ch->cap, ch->side);
        ch->cur_p ^= 1;
        launch_reconnect(ch->vp, d, ch->cur_p, ch->cap, point_span(ch->n_hint, ch->cap), ch->hsize, ch->side);
        ch->cur_p ^= 1;
        if (s + 1 < nst) {
            if (pre) vfm_pre(ch, ch->side);
            cudaStreamWaitEvent(ch->side, ch->ev_join, 0);
        }
    }
    cudaEventRecord(ch->ev_join, ch->side);
    cudaStreamWaitEvent(ch->stream, ch->ev_join, 0);
}

// Replay `multi ? GRAPH_MULTI : 1` coupled steps from a graph captured on
// first use for the current buffer parities and filament size class.
bool step_graph(vlb_channel* ch, bool multi) {
    const int m = multi ? 1 : 0, nst = multi ? GRAPH_MULTI : 1;
    const int f = ch->cur_f, q = ch->cur_p;
    const int cls = size_class(ch->n_hint);
    cudaGraphExec_t& ge = ch->gexec[m][f][q];
    const bool f_clean0 = ch->f_clean;
    auto undo = [&] {  // nothing ran: back to the state before the attempt
        ch->cur_f = f;
        ch->cur_p = q;
        ch->f_clean = f_clean0;
        return false;
    };
    if (ge && ch->gclass[m][f][q] != cls) {
        // the Biot-Savart grid was sized for another filament count: capture again
        cudaGraphExecDestroy(ge);
        ge = nullptr;
    }
    if (!ge) {
        cudaGraph_t graph = nullptr;
        const bool forked = nst > 1 && ch->overlap && ensure_side(ch);  // before the capture begins
        if (cudaStreamBeginCapture(ch->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return undo();
        }
        tl_no_pdl = true;
        if (forked) run_steps_forked(ch, nst);
        else
            for (int k = 0; k < nst; ++k) run_phases(ch, VLB_PHASE_ALL);
        tl_no_pdl = false;
        cudaError_t e = cudaStreamEndCapture(ch->stream, &graph);
        ch->cur_f = f;  // the captured steps have not run yet
        ch->cur_p = q;
        if (e != cudaSuccess || !graph) {
            cudaGetLastError();
            return undo();
        }
        e = cudaGraphInstantiate(&ge, graph, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ge = nullptr;
            return undo();
        }
        ch->gclass[m][f][q] = cls;
    }
    if (cudaGraphLaunch(ge, ch->stream) != cudaSuccess) return undo();
    if (nst & 1) ch->cur_f ^= 1;  // the point buffers are back to q after remesh and reconnect
    ch->f_clean = !ch->p.couple;  // state after full steps: the last one spread its reaction
    return true;
}

// Capture body() on stream s as split graph kind/par if it is missing or
// was sized for another filament count; nothing is launched.  body() runs on
// the channel's state as it will be at launch and leaves it as it found it.
bool capture_split(vlb_channel* ch, int kind, int par, cudaStream_t s, const std::function<void()>& body) {
    const int cls = size_class(ch->n_hint);
    cudaGraphExec_t& ge = ch->sgexec[kind][par];
    if (ge && ch->sgclass[kind][par] == cls) return true;
    if (ge) cudaGraphExecDestroy(ge);
    ge = nullptr;
    const int f = ch->cur_f, q = ch->cur_p;
    const bool fc = ch->f_clean;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    tl_no_pdl = true;
    body();
    tl_no_pdl = false;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    ch->cur_f = f;
    ch->cur_p = q;
    ch->f_clean = fc;
    if (e != cudaSuccess || !graph) {
        cudaGetLastError();
        return false;
    }
    e = cudaGraphInstantiate(&ge, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ge = nullptr;
        return false;
    }
    ch->sgclass[kind][par] = cls;
    return true;
}

// One coupled step of vlb_step_async, split over the two streams:
//   channel stream: lattice pass (v_n in every tile, its mass and Mach into
//     the parity slot DS_LAT + 2 f), then, once the second stream's work of
//     the previous split step is done, the RK stages;
//   second stream: after the stages, remesh, reconnection, the line length
//     and the status copy into the call's pinned slot.
// The lattice pass of the next call then runs beside this call's remesh and
// reconnection, as in the overlapped multi-step graphs, with the same result
// bit for bit.  False, with nothing queued, if it cannot be set up; the call
// then queues the step in sequence.
bool queue_split_step(vlb_channel* ch, int slot) {
    if (!(ch->graphs && !ch->timing && ch->stream && ch->overlap && ensure_side(ch))) return false;
    if ((!ch->ev_a && cudaEventCreateWithFlags(&ch->ev_a, cudaEventDisableTiming) != cudaSuccess) ||
        (!ch->ev_b && cudaEventCreateWithFlags(&ch->ev_b, cudaEventDisableTiming) != cudaSuccess)) {
        cudaGetLastError();
        return false;
    }
    Dev& d = ch->d;
    cudaStream_t A = ch->stream, B = ch->side;
    const int f = ch->cur_f, q = ch->cur_p;
    auto lat = [&] { lattice_pass(ch, true, d.dstats + DS_LAT + 2 * f); };
    auto stages = [&] {
        ch->f_clean = true;  // the lattice pass before consumed the force grid
        vfm_step(ch, false, A);
    };
    auto topo = [&] {
        const int span = point_span(ch->n_hint, ch->cap);
        launch_remesh(ch->vp, d, ch->cur_p, ch->cap, span, B);
        ch->cur_p ^= 1;
        launch_reconnect(ch->vp, d, ch->cur_p, ch->cap, span, ch->hsize, B);
        ch->cur_p ^= 1;
        launch_line_length(ch->lp.g, d.pos[ch->cur_p], d.next[ch->cur_p], d.counters, ch->cap, d.line_part,
                           d.dstats, B);
    };
    if (!capture_split(ch, 0, f, A, lat) || !capture_split(ch, 1, q, A, stages) || !capture_split(ch, 2, q, B, topo))
        return false;
    // this lattice pass writes the parity slot of the call two back: its status copy must be done
    if (ch->q_head >= 2) cudaStreamWaitEvent(A, ch->q_ev[(ch->q_head - 2) % VLB_ASYNC_DEPTH], 0);
    if (cudaGraphLaunch(ch->sgexec[0][f], A) != cudaSuccess) return false;
    if (ch->b_tail) cudaStreamWaitEvent(A, ch->ev_b, 0);
    cudaGraphLaunch(ch->sgexec[1][q], A);
    cudaEventRecord(ch->ev_a, A);
    cudaStreamWaitEvent(B, ch->ev_a, 0);
    cudaGraphLaunch(ch->sgexec[2][q], B);
    cudaEventRecord(ch->ev_b, B);  // the points are final: the next call's stages may start
    cudaMemcpyAsync(ch->h_ring + (size_t)slot * STATUS_SLOT, d.dstats, STATUS_BYTES, cudaMemcpyDeviceToHost, B);
    cudaEventRecord(ch->q_ev[slot], B);
    ch->b_tail = true;
    ch->b_slot = slot;
    ch->last_lat = f;
    ch->cur_f ^= 1;
    ch->f_clean = !ch->p.couple;
    ch->steps++;
    return true;
}

// Queue nsteps coupled steps: multi-step graphs while enough steps remain,
// then single-step graphs; direct launches when graphs are off or unavailable.
void queue_steps(vlb_channel* ch, int nsteps) {
    const bool use_graph = ch->graphs && !ch->timing && ch->stream != nullptr;
    int k = 0;
    while (k < nsteps) {
        if (use_graph && nsteps - k >= GRAPH_MULTI && step_graph(ch, true)) {
            k += GRAPH_MULTI;
            ch->steps += GRAPH_MULTI;
            continue;
        }
        if (!(use_graph && step_graph(ch, false))) run_phases(ch, VLB_PHASE_ALL);
        ++k;
        ch->steps++;
    }
}
}  // namespace

namespace {
// The STATS record (VLB_FIELD_STATS) from a status block.
// lat >= 0: the mass and Mach come from that parity slot of a split step.
void fill_stats(const vlb_channel* ch, const double* ds, const int* cnt, long long steps, double* o, int lat = -1) {
    const double* m = lat >= 0 ? ds + DS_LAT + 2 * lat : ds + DS_MASS;
    for (int k = 0; k < 16; ++k) o[k] = 0.0;
    o[0] = cnt[CNT_N];
    o[1] = cnt[CNT_STATUS];
    o[2] = m[0];
    o[3] = ds[DS_LINE];
    o[4] = m[1];
    o[5] = ds[DS_SPLITS];
    o[6] = ds[DS_MERGES];
    o[7] = ds[DS_RECON];
    o[8] = ds[DS_SMALL];
    o[9] = (double)steps;
    o[10] = (double)ch->bytes;
    o[13] = ds[DS_WALLCUT];
}
}  // namespace

int vlb_step(vlb_channel* ch, int32_t nsteps) {
    if (!ch || nsteps < 0) return fail(VLB_ERR_INVALID_ARG, "bad step arguments");
    if (ch->q_head != ch->q_tail) return fail(VLB_ERR_INVALID_ARG, "vlb_step_async calls still queued");
    join_side(ch);
    ch->line_fresh = false;
    queue_steps(ch, nsteps);
    // the total line length of the new points rides along with the status read,
    // so a vlb_line_length right after the steps needs no launch or wait of its own
    if (nsteps > 0)
        launch_line_length(ch->lp.g, ch->d.pos[ch->cur_p], ch->d.next[ch->cur_p], ch->d.counters, ch->cap,
                           ch->d.line_part, ch->d.dstats, ch->stream);
    const int rc = finish(ch);
    ch->line_fresh = rc == VLB_OK && nsteps > 0;
    return rc;
}

int vlb_step_async(vlb_channel* ch, int32_t nsteps) {
    if (!ch || nsteps < 0) return fail(VLB_ERR_INVALID_ARG, "bad step arguments");
    if (ch->q_head - ch->q_tail >= VLB_ASYNC_DEPTH)
        return fail(VLB_ERR_INVALID_ARG, "VLB_ASYNC_DEPTH calls already queued: complete one with vlb_query");
    const int slot = ch->q_head % VLB_ASYNC_DEPTH;
    if (!ch->q_ev[slot] && cudaEventCreateWithFlags(&ch->q_ev[slot], cudaEventDisableTiming) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "event create");
    if (!ch->h_ring && cudaMallocHost((void**)&ch->h_ring, STATUS_SLOT * VLB_ASYNC_DEPTH) != cudaSuccess) {
        ch->h_ring = nullptr;
        return fail(VLB_ERR_OOM, "pinned status slots");
    }
    ch->line_fresh = false;
    ch->q_lat[slot] = -1;
    if (nsteps == 1 && queue_split_step(ch, slot)) {
        ch->q_lat[slot] = ch->last_lat;
    } else {
        join_side(ch);
        queue_steps(ch, nsteps);
        if (nsteps > 0)  // as in vlb_step: the line length of the new points rides along with the status
            launch_line_length(ch->lp.g, ch->d.pos[ch->cur_p], ch->d.next[ch->cur_p], ch->d.counters, ch->cap,
                               ch->d.line_part, ch->d.dstats, ch->stream);
        cudaMemcpyAsync(ch->h_ring + (size_t)slot * STATUS_SLOT, ch->d.dstats, STATUS_BYTES, cudaMemcpyDeviceToHost,
                        ch->stream);
        cudaEventRecord(ch->q_ev[slot], ch->stream);
    }
    ch->q_line[slot] = nsteps > 0;
    ch->q_steps[slot] = ch->steps;
    ++ch->q_head;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "step launch");
    return VLB_OK;
}

int vlb_query(vlb_channel* ch) {
    if (!ch) return fail(VLB_ERR_INVALID_ARG, "null channel");
    if (ch->q_head == ch->q_tail) return VLB_OK;
    const int slot = ch->q_tail % VLB_ASYNC_DEPTH;
    const cudaError_t e = cudaEventQuery(ch->q_ev[slot]);
    if (e == cudaErrorNotReady) return VLB_BUSY;
    ++ch->q_tail;
    if (e != cudaSuccess) return cuda_fail(e, "step completion");
    // this call's status block: kept for vlb_query_stats, and the channel's
    // host copy of the status until the state is read again
    memcpy(ch->done_block, ch->h_ring + (size_t)slot * STATUS_SLOT, STATUS_BYTES);
    ch->done_steps = ch->q_steps[slot];
    ch->done_lat = ch->q_lat[slot];
    memcpy(ch->h_dstats, ch->done_block, STATUS_BYTES);
    ch->n_hint = ch->h_counters[CNT_N];
    ch->line_fresh = ch->q_line[slot] && ch->q_head == ch->q_tail;
    std::string msg;
    const int rc = status_to_code(ch->h_counters[CNT_STATUS], &msg);
    if (rc) {
        ch->line_fresh = false;
        return fail(rc, msg);
    }
    return VLB_OK;
}

int vlb_query_stats(vlb_channel* ch, double* out) {
    if (!ch || !out) return fail(VLB_ERR_INVALID_ARG, "null argument");
    if (ch->done_steps < 0) return fail(VLB_ERR_INVALID_ARG, "no vlb_step_async call has completed");
    fill_stats(ch, (const double*)ch->done_block, (const int*)(ch->done_block + sizeof(double) * DS_COUNT),
               ch->done_steps, out, ch->done_lat);
    return VLB_OK;
}

int vlb_set_graphs(vlb_channel* ch, int32_t enable) {
    if (!ch) return fail(VLB_ERR_INVALID_ARG, "null channel");
    ch->graphs = enable != 0;
    return VLB_OK;
}

int vlb_set_overlap(vlb_channel* ch, int32_t enable) {
    if (!ch) return fail(VLB_ERR_INVALID_ARG, "null channel");
    if (ch->q_head != ch->q_tail) return fail(VLB_ERR_INVALID_ARG, "steps still queued");
    join_side(ch);
    if (ch->overlap != (enable != 0)) {
        // the multi-step graphs were captured in the other form
        cudaStreamSynchronize(ch->stream);
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                if (ch->gexec[1][a][b]) {
                    cudaGraphExecDestroy(ch->gexec[1][a][b]);
                    ch->gexec[1][a][b] = nullptr;
                    ch->gclass[1][a][b] = -1;
                }
    }
    ch->overlap = enable != 0;
    return VLB_OK;
}

int vlb_run_phases(vlb_channel* ch, int32_t mask) {
    if (!ch || mask < 0 || mask > VLB_PHASE_ALL) return fail(VLB_ERR_INVALID_ARG, "bad phase mask");
    join_side(ch);
    ch->line_fresh = false;
    run_phases(ch, mask);
    return finish(ch);
}

int vlb_read_fields(vlb_channel* ch, int32_t which, void* dst, size_t bytes, size_t* written) {
    if (!ch || !dst) return fail(VLB_ERR_INVALID_ARG, "null argument");
    int rc = sync_counters(ch);
    if (rc) return rc;
    const long long C = ch->lp.g.ncell;
    const int N = ch->h_counters[CNT_N];
    size_t need = 0;
    switch (which) {
        case VLB_FIELD_RHO: need = sizeof(float) * (size_t)C; break;
        case VLB_FIELD_U: case VLB_FIELD_FORCE: need = sizeof(float) * 3 * (size_t)C; break;
        case VLB_FIELD_FSTAR: case VLB_FIELD_FDEV: need = sizeof(float) * 19 * (size_t)C; break;
        case VLB_FIELD_POS: case VLB_FIELD_VEL: need = sizeof(double) * 3 * (size_t)N; break;
        case VLB_FIELD_NEXT: need = sizeof(int) * (size_t)N; break;
        case VLB_FIELD_PLANE_VS: case VLB_FIELD_LINE_PROFILE: need = sizeof(double) * (size_t)ch->lp.g.nz; break;
        case VLB_FIELD_STATS: need = sizeof(double) * 16; break;
        default: return fail(VLB_ERR_INVALID_ARG, "unknown field");
    }
    if (bytes < need) return fail(VLB_ERR_INVALID_ARG, "destination buffer too small");
    Dev& d = ch->d;
    cudaStream_t s = ch->stream;
    float* tmp = (float*)d.f[ch->cur_f ^ 1];  // scratch between steps
    const int esize = ch->p.storage == VLB_STORE_F32 ? 4 : 2;
    const int per_chunk = (int)((19 * (size_t)esize) / 4);  // populations per float chunk the spare buffer holds
    cudaError_t e = cudaSuccess;
    if (which == VLB_FIELD_RHO || which == VLB_FIELD_U) {
        launch_moments(ch->lp, d.f[ch->cur_f], d.F, d.fmask, tmp, tmp + C, s);
        e = cudaMemcpyAsync(dst, which == VLB_FIELD_RHO ? tmp : tmp + C, need, cudaMemcpyDeviceToHost, s);
    } else if (which == VLB_FIELD_FSTAR || which == VLB_FIELD_FDEV) {
        for (int i0 = 0; i0 < 19 && e == cudaSuccess; i0 += per_chunk) {
            const int i1 = i0 + per_chunk < 19 ? i0 + per_chunk : 19;
            launch_export(ch->lp, d.f[ch->cur_f], tmp, i0, i1, which == VLB_FIELD_FSTAR ? +1 : 0, s);
            e = cudaMemcpyAsync((char*)dst + sizeof(float) * (size_t)i0 * C, tmp, sizeof(float) * (size_t)(i1 - i0) * C,
                                cudaMemcpyDeviceToHost, s);
        }
    } else if (which == VLB_FIELD_FORCE) {
        launch_force_export(ch->lp.g, d.F, tmp, s);  // spare population buffer holds 12 B per cell
        e = cudaMemcpyAsync(dst, tmp, need, cudaMemcpyDeviceToHost, s);
    } else if (which == VLB_FIELD_POS || which == VLB_FIELD_VEL) {
        std::vector<double> soa(3 * (size_t)ch->cap);
        const double* src = which == VLB_FIELD_POS ? d.pos[ch->cur_p] : d.vel1;
        e = cudaMemcpyAsync(soa.data(), src, sizeof(double) * 3 * (size_t)ch->cap, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "read positions");
        double* o = (double*)dst;
        for (int i = 0; i < N; ++i)
            for (int a = 0; a < 3; ++a) o[3 * (size_t)i + a] = soa[(size_t)a * ch->cap + i];
    } else if (which == VLB_FIELD_NEXT) {
        if (N > 0) e = cudaMemcpyAsync(dst, d.next[ch->cur_p], need, cudaMemcpyDeviceToHost, s);
    } else if (which == VLB_FIELD_PLANE_VS) {
        e = cudaMemcpyAsync(dst, d.Vs, need, cudaMemcpyDeviceToHost, s);
    } else if (which == VLB_FIELD_LINE_PROFILE) {
        double* prof = (double*)tmp;  // spare population buffer
        launch_line_profile(ch->lp.g, d.pos[ch->cur_p], d.next[ch->cur_p], d.counters, ch->cap, prof, s);
        e = cudaMemcpyAsync(dst, prof, need, cudaMemcpyDeviceToHost, s);
    } else {
        launch_line_length(ch->lp.g, d.pos[ch->cur_p], d.next[ch->cur_p], d.counters, ch->cap, d.line_part, d.dstats, s);
        rc = sync_counters(ch);
        if (rc) return rc;
        fill_stats(ch, ch->h_dstats, ch->h_counters, ch->steps, (double*)dst);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "read field");
    if (written) *written = need;
    return VLB_OK;
}

int vlb_write_fields(vlb_channel* ch, int32_t which, const void* src, size_t bytes) {
    if (!ch || !src) return fail(VLB_ERR_INVALID_ARG, "null argument");
    join_side(ch);
    ch->line_fresh = false;
    const long long C = ch->lp.g.ncell;
    Dev& d = ch->d;
    cudaStream_t s = ch->stream;
    cudaError_t e;
    if (which == VLB_FIELD_FSTAR) {
        if (bytes != sizeof(float) * 19 * (size_t)C) return fail(VLB_ERR_INVALID_ARG, "FSTAR size mismatch");
        float* tmp = (float*)d.f[ch->cur_f ^ 1];
        const int esize = ch->p.storage == VLB_STORE_F32 ? 4 : 2;
        const int per_chunk = (int)((19 * (size_t)esize) / 4);
        e = cudaSuccess;
        for (int i0 = 0; i0 < 19 && e == cudaSuccess; i0 += per_chunk) {
            const int i1 = i0 + per_chunk < 19 ? i0 + per_chunk : 19;
            e = cudaMemcpyAsync(tmp, (const char*)src + sizeof(float) * (size_t)i0 * C,
                                sizeof(float) * (size_t)(i1 - i0) * C, cudaMemcpyHostToDevice, s);
            launch_import(ch->lp, tmp, d.f[ch->cur_f], i0, i1, s);
        }
    } else if (which == VLB_FIELD_FORCE) {
        if (bytes != sizeof(float) * 3 * (size_t)C) return fail(VLB_ERR_INVALID_ARG, "FORCE size mismatch");
        float* tmp = (float*)d.f[ch->cur_f ^ 1];  // spare population buffer
        e = cudaMemcpyAsync(tmp, src, bytes, cudaMemcpyHostToDevice, s);
        launch_force_import(ch->lp.g, tmp, d.F, s);
        ch->f_clean = false;
        const int nt = ch->lp.g.tnx * ch->lp.g.tny * ch->lp.g.tnz;
        cudaMemsetAsync(d.fmask, 1, (size_t)nt, s);
    } else {
        return fail(VLB_ERR_INVALID_ARG, "field is not writable");
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "write field");
    return VLB_OK;
}

int vlb_line_length(vlb_channel* ch, double* out) {
    if (!ch || !out) return fail(VLB_ERR_INVALID_ARG, "null argument");
    if (ch->line_fresh) {  // computed at the end of the last vlb_step
        *out = ch->h_dstats[DS_LINE];
        return VLB_OK;
    }
    join_side(ch);
    launch_line_length(ch->lp.g, ch->d.pos[ch->cur_p], ch->d.next[ch->cur_p], ch->d.counters, ch->cap,
                       ch->d.line_part, ch->d.dstats, ch->stream);
    cudaMemcpyAsync(ch->h_dstats + DS_LINE, ch->d.dstats + DS_LINE, sizeof(double), cudaMemcpyDeviceToHost,
                    ch->stream);
    cudaError_t e = cudaStreamSynchronize(ch->stream);
    if (e != cudaSuccess) return cuda_fail(e, "line length");
    *out = ch->h_dstats[DS_LINE];
    return VLB_OK;
}

int vlb_set_timing(vlb_channel* ch, int32_t enable) {
    if (!ch) return fail(VLB_ERR_INVALID_ARG, "null channel");
    join_side(ch);
    cudaStreamSynchronize(ch->stream);
    ch->timing = enable != 0;
    for (int k = 0; k < VLB_TIMED_KINDS; ++k) {
        ch->ev_used[k] = 0;
        ch->timing_ms[k] = 0.0;
        ch->timing_launches[k] = 0;
    }
    return VLB_OK;
}

int vlb_kernel_timing(vlb_channel* ch, int32_t kind, double* total_ms, int64_t* launches) {
    if (!ch || !total_ms || !launches) return fail(VLB_ERR_INVALID_ARG, "null argument");
    if (kind < 0 || kind >= VLB_TIMED_KINDS) return fail(VLB_ERR_INVALID_ARG, "unknown timed kernel kind");
    cudaError_t e = cudaStreamSynchronize(ch->stream);
    if (e != cudaSuccess) return cuda_fail(e, "timing sync");
    std::vector<cudaEvent_t>& list = ch->ev[kind];
    for (size_t k = 0; k + 1 < ch->ev_used[kind]; k += 2) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, list[k], list[k + 1]);
        ch->timing_ms[kind] += ms;
        ch->timing_launches[kind]++;
    }
    ch->ev_used[kind] = 0;
    *total_ms = ch->timing_ms[kind];
    *launches = ch->timing_launches[kind];
    return VLB_OK;
}

int vlb_lbm_timing(vlb_channel* ch, double* total_ms, int64_t* launches) {
    return vlb_kernel_timing(ch, VLB_TIMED_LBM, total_ms, launches);
}

size_t vlb_biot_savart_scratch_bytes(int32_t n) { return bs_scratch_bytes(n < 1 ? 1 : n); }

int vlb_biot_savart(const vlb_params* p, const double* pos, const int32_t* next, int32_t n, float* vel, void* scratch,
                    size_t scratch_bytes, void* stream) {
    return vlb::bs_standalone(p, pos, next, n, vel, scratch, scratch_bytes, stream);
}

}  // extern "C"
