// Vortex-filament part of the coupled step (Sec. II.A of arXiv 2108.04435)
// and the coupling exchange (Eqs. 10-11): per-point geometry and the local
// self-induced term, the equation of motion (Eq. 4) with RK4 staging, the
// 2-point-delta interpolation of v_n and the spreading of the friction
// reaction onto the lattice.
//
// The FP64 geometry that feeds the remeshing decisions lives in topo.cu.
#include <cuda_runtime.h>
#include <math.h>

#include "eom.cuh"
#include "records.cuh"
#include "vlb_internal.cuh"

namespace vlb {

namespace {

// Stage geometry of point i for the equation of motion: the same quantities as
// k_geometry (remeshing decisions use that FP64 kernel instead), stored as
// float for the FP32 equation of motion and Biot-Savart sum.  An open end pinned on a wall takes the mirror image
// of its neighbour across that wall as its missing neighbour, represents half
// of its segment, and carries its wall code (+1) to the equation of motion; a
// line's last point starts no segment.  The source slots go where the slots
// of the order o put them.
struct StageRec {
    int p, q;      // predecessor and successor, -1 at a line's first / last point
    int pin;       // wall code of a pinned end, -1 otherwise
    double si[3];  // the point
    double st[3];  // its successor (itself at a line's last point)
    float b[3];    // the segment (zero at a line's last point)
};

__device__ __forceinline__ void geometry_point(const VfmParams& P, const double* __restrict__ s,
                                               const int* __restrict__ next, const int* __restrict__ prev, int N,
                                               int cap, int i, float4* __restrict__ geo, double* __restrict__ s0_copy,
                                               StageRec& out) {
    const int p = prev[i], q = next[i];
    const int pl = p >= 0 ? p : i, ql = q >= 0 ? q : i;  // an end loads itself in place of the missing one
    double si[3], sp[3], sq[3];
    float b[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        si[k] = s[(long long)k * cap + i];
        sp[k] = s[(long long)k * cap + pl];
        sq[k] = s[(long long)k * cap + ql];
    }
    int code = -1;
    if (p < 0 || q < 0) {
        code = touching_wall(P.g, P.dmin, si);
        const int ax = code >> 1;
        const double L = (double)(ax == 0 ? P.g.nx : (ax == 1 ? P.g.ny : P.g.nz));
        const double w2 = 2.0 * ((code & 1) ? L - 0.5 : -0.5);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double nb = p < 0 ? sq[k] : sp[k];
            // mirror image across the wall; an end on no wall is continued straight
            const double g = code < 0 ? 2.0 * si[k] - nb : (k == ax ? w2 - nb : nb);
            if (p < 0) sp[k] = g;
            else sq[k] = g;
        }
    }
    // Neighbour differences a = s_i - s_p, b = s_q - s_i in FP64 (positions
    // are up to ~1e3 cells).  With the 3-point derivatives on the non-uniform
    // grid, s' = (l-^2 b + l+^2 a) / D and s'' = 2 (l- b - l+ a) / D,
    // D = l+ l- (l+ + l-), the local term beta s' x s'' is exactly
    // 2 beta (a x b) / D.  Its near-singular part is a x b: on a gently curved
    // line a and b are nearly parallel and their cross product cancels, so it
    // is formed in FP64; the lengths, beta and 1/D are smooth and stay FP32
    // (relative error ~1e-7).
    double da[3], db[3];
    float a[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (s0_copy) s0_copy[(long long)k * cap + i] = si[k];  // first stage: RK4 base positions
        da[k] = min_image(P.g, k, si[k] - sp[k]);
        db[k] = min_image(P.g, k, sq[k] - si[k]);
        a[k] = (float)da[k];
        b[k] = (float)db[k];
    }
    const float lm = sqrtf(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    const float lp = sqrtf(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    const float inv = 1.f / (lp * lm * (lp + lm));
    float t1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) t1[k] = (lm * lm * b[k] + lp * lp * a[k]) * inv;
    const double ab[3] = {da[1] * db[2] - da[2] * db[1], da[2] * db[0] - da[0] * db[2], da[0] * db[1] - da[1] * db[0]};
    // beta = kappa/4pi ln(2 sqrt(l+ l-) / (e^{1/4} a)) = kappa/4pi (C + ln(l+ l-) / 2), C = ln(2 / (e^{1/4} a))
    const float beta = P.kq_f * (P.beta_c_f + 0.5f * logf(lp * lm));
    const float fl = 2.f * beta * inv;
    // geo[2i] = (s'.xyz, dxi), geo[2i+1] = (local velocity beta s' x s'', wall code + 1 of a pinned end)
    const float dxi = p < 0 ? 0.5f * lp : (q < 0 ? 0.5f * lm : 0.5f * (lp + lm));
    geo[2LL * i] = make_float4(t1[0], t1[1], t1[2], dxi);
    geo[2LL * i + 1] = make_float4(fl * (float)ab[0], fl * (float)ab[1], fl * (float)ab[2], (float)(code + 1));
    if (q < 0) b[0] = b[1] = b[2] = 0.f;  // no segment leaves a line's last point
    out.p = p;
    out.q = q;
    out.pin = code;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        out.si[a] = si[a];
        out.st[a] = q >= 0 ? sq[a] : si[a];  // a line's last point starts no segment: its image is zero-length
        out.b[a] = b[a];
    }
}

// One block per group of source slots, thread t for slot t of the group:
// the slot's point (its stage geometry, its target record and its slot), a
// gap slot's copy of a successor, or a zero padding slot; the group's
// records of every record block then go out together (records.cuh).
// Block 0 also resets the work counter of the Biot-Savart launch that
// follows.
__global__ void __launch_bounds__(BS_GROUP) k_geometry_stage(VfmParams P, const double* __restrict__ s,
                                                             const int* __restrict__ next,
                                                             const int* __restrict__ prev,
                                                             int* __restrict__ counters, int cap,
                                                             float4* __restrict__ geo, float4* __restrict__ seg,
                                                             double* __restrict__ s0_copy, BsOrder o) {
    pdl_wait_trigger();
    __shared__ BsGroupSmem sm;
    const int N = counters[CNT_N];
    const int ns = counters[CNT_NSLOT];
    const long long Np = bs_block(ns);
    if (blockIdx.x == 0 && threadIdx.x == 0) counters[CNT_BSWORK] = 0;  // the Biot-Savart launch takes items from 0
    const int ng = (int)(Np / BS_GROUP);
    for (int grp = blockIdx.x; grp < ng; grp += gridDim.x) {
        const int sl = grp * BS_GROUP + threadIdx.x;
        const int code = sl < ns ? o.pt[sl] : -1;
        int4 og = o.org[grp];
        const double O[3] = {(double)og.x, (double)og.y, (double)og.z};
        double rel[3] = {0.0, 0.0, 0.0};
        float d[3] = {0.f, 0.f, 0.f};
        bool jump = false;
        int prev_sl = -1, excl = -1;
        if (code >= 0) {
            StageRec r;
            geometry_point(P, s, next, prev, N, cap, code, geo, s0_copy, r);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                rel[a] = min_image(P.g, a, r.si[a] - O[a]);
                d[a] = r.b[a];
                // the next slot of the group holds the successor at min_image(s_q - O)
                if (r.q >= 0 && threadIdx.x != BS_GROUP - 1)
                    jump |= fabs(min_image(P.g, a, r.st[a] - O[a]) - (rel[a] + (double)r.b[a])) > 0.5;
            }
            prev_sl = bs_prev_slot(o, r.p);
            for (int f = 0; f < P.nfaces; ++f)
                if (r.pin >= 0 && P.face_code[f] == r.pin) excl = (int)((1 + f) * Np) + (r.p < 0 ? sl : prev_sl);
        } else if (code <= -2) {
            const int q = next[-2 - code];
#pragma unroll
            for (int a = 0; a < 3; ++a) rel[a] = min_image(P.g, a, s[(long long)a * cap + q] - O[a]);
        }
        if (s0_copy) {
            // the first stage of the step: the origin moves to the centre of the group's box
            og = bs_center_origin(rel, og, sm);
            if (threadIdx.x == 0) o.org[grp] = og;
        }
        if (code >= 0) bs_write_target(o.tgt, o.sorted ? o.rank[code] : code, rel, og, sl, prev_sl, excl, code);
        bs_write_group(P.nfaces, P.face_code, Np, grp, rel, d, jump, seg, sm);
    }
}

// The equation of motion of each point as a kernel of its own (used when the
// Biot-Savart pass does not apply it).
__global__ void __launch_bounds__(64) k_eom(EomArgs A, const float* __restrict__ vbs, long long* __restrict__ vacc) {
    pdl_wait_trigger();
    const int N = A.counters[CNT_N];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < N;
    float v[3] = {0.f, 0.f, 0.f};
    if (valid) {
        if (vacc) {
            for (int k = 0; k < 3; ++k) {
                v[k] = bs_value(vacc[(long long)k * A.cap + i]);
                vacc[(long long)k * A.cap + i] = 0;  // cleared for the next Biot-Savart pass
            }
        } else {
            for (int k = 0; k < 3; ++k) v[k] = vbs[(long long)k * A.cap + i];
        }
    }
    eom_point(A, i, valid, v[0], v[1], v[2]);
}

// Total line length sum |s_next(i) - s_i| (FP64): per-block sums in a fixed
// order, the last block to finish adds the block sums in block order.
__global__ void __launch_bounds__(256) k_line_length(Grid g, const double* __restrict__ pos,
                                                      const int* __restrict__ next, int* __restrict__ counters,
                                                      int cap, double* __restrict__ part, double* __restrict__ dstats) {
    pdl_wait_trigger();
    __shared__ double sm[256];
    __shared__ int s_last;
    const int N = counters[CNT_N];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (i < N && next[i] >= 0) {
        const int q = next[i];
        double d[3];
        for (int k = 0; k < 3; ++k) d[k] = min_image(g, k, pos[(long long)k * cap + q] - pos[(long long)k * cap + i]);
        v = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    }
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = sm[0];
        __threadfence();
        s_last = atomicAdd(&counters[CNT_LINEDONE], 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double acc = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) acc += __ldcg(&part[k]);
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        dstats[DS_LINE] = sm[0];
        counters[CNT_LINEDONE] = 0;
    }
}

// Line length per z plane: each segment's length goes to the plane nearest
// its midpoint (periodic z wraps, walls clamp); FP64 atomics.
__global__ void k_line_profile(Grid g, const double* __restrict__ pos, const int* __restrict__ next,
                               const int* __restrict__ counters, int cap, double* __restrict__ prof) {
    const int N = counters[CNT_N];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int q = next[i];
    if (q < 0) return;
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = min_image(g, k, pos[(long long)k * cap + q] - pos[(long long)k * cap + i]);
    const double mid = pos[2LL * cap + i] + 0.5 * d[2];
    int k = (int)floor(mid + 0.5);
    if (!g.wall[2]) k = ((k % g.nz) + g.nz) % g.nz;
    else k = k < 0 ? 0 : (k > g.nz - 1 ? g.nz - 1 : k);
    atomicAdd(&prof[k], sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
}

}  // namespace

void launch_geometry_stage(const VfmParams& P, const double* s, const int* next, const int* prev, int* counters,
                           int cap, int span, float4* geo, float4* seg, double* s0_copy, const BsOrder& o,
                           cudaStream_t st) {
    if (cap <= 0) return;
    launch_pdl(k_geometry_stage, (int)(bs_slot_cap(span) / BS_GROUP), BS_GROUP, 0, st, P, s, next, prev, counters,
               cap, geo, seg, s0_copy, o);
}

void launch_eom(const EomArgs& A, const float* vbs, cudaStream_t s, long long* vacc) {
    if (A.cap <= 0) return;
    launch_pdl(k_eom, (A.cap + 63) / 64, 64, 0, s, A, vbs, vacc);
}

void launch_line_length(const Grid& g, const double* pos, const int* next, int* counters, int cap, double* part,
                        double* dstats, cudaStream_t s) {
    launch_pdl(k_line_length, (cap + 255) / 256, 256, 0, s, g, pos, next, counters, cap, part, dstats);
}

void launch_line_profile(const Grid& g, const double* pos, const int* next, const int* counters, int cap,
                         double* prof, cudaStream_t s) {
    cudaMemsetAsync(prof, 0, sizeof(double) * (size_t)g.nz, s);
    if (cap > 0) k_line_profile<<<(cap + 255) / 256, 256, 0, s>>>(g, pos, next, counters, cap, prof);
}

}  // namespace vlb
