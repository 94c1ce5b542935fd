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
#include "vlb_internal.cuh"

namespace vlb {

namespace {


// Stage geometry for the equation of motion: the same quantities as
// k_geometry, with the neighbour differences formed in FP64 (positions are up
// to ~1e3 cells) and everything after them in FP32, which is accurate to
// ~1e-7 relative for segments of O(1) cells.  The remeshing decisions use the
// FP64 k_geometry instead.  An open end pinned on a wall takes the mirror image
// of its neighbour across that wall as its missing neighbour, represents half
// of its segment, and carries its wall code (+1) to the equation of motion; a
// line's last point has a zero-length source record.
__global__ void __launch_bounds__(64) k_geometry_stage(VfmParams P, const double* __restrict__ s,
                                                       const int* __restrict__ next, const int* __restrict__ prev,
                                                       int* __restrict__ counters, int cap,
                                                       float4* __restrict__ geo, float4* __restrict__ seg,
                                                       double* __restrict__ s0_copy) {
    pdl_wait_trigger();
    const int N = counters[CNT_N];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) counters[CNT_BSWORK] = 0;  // the Biot-Savart launch that follows takes items from 0
    if (i >= N) return;
    const int p = prev[i], q = next[i];
    const int pl = p >= 0 ? p : i, ql = q >= 0 ? q : i;  // an end loads itself in place of the missing one
    double si[3], sp[3], sq[3];
    float a[3], b[3];
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
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (s0_copy) s0_copy[(long long)k * cap + i] = si[k];  // first stage: RK4 base positions
        a[k] = (float)min_image(P.g, k, si[k] - sp[k]);
        b[k] = (float)min_image(P.g, k, sq[k] - si[k]);
    }
    const float lm = sqrtf(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    const float lp = sqrtf(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    const float inv = 1.f / (lp * lm * (lp + lm));
    float t1[3], t2[3];
    for (int k = 0; k < 3; ++k) {
        t1[k] = (lm * lm * b[k] + lp * lp * a[k]) * inv;
        t2[k] = 2.f * (lm * b[k] - lp * a[k]) * inv;
    }
    const float beta = P.kq_f * logf(2.f * sqrtf(lp * lm) * P.inv_ea_f);
    // geo[2i] = (s'.xyz, dxi), geo[2i+1] = (local velocity beta s' x s'', wall code + 1 of a pinned end)
    const float dxi = p < 0 ? 0.5f * lp : (q < 0 ? 0.5f * lm : 0.5f * (lp + lm));
    geo[2LL * i] = make_float4(t1[0], t1[1], t1[2], dxi);
    geo[2LL * i + 1] = make_float4(beta * (t1[1] * t2[2] - t1[2] * t2[1]), beta * (t1[2] * t2[0] - t1[0] * t2[2]),
                                   beta * (t1[0] * t2[1] - t1[1] * t2[0]), (float)(code + 1));
    if (q < 0) b[0] = b[1] = b[2] = 0.f;  // no segment leaves a line's last point
    float hi[3], lo[3];
    for (int k = 0; k < 3; ++k) {
        hi[k] = __double2float_rn(si[k]);
        lo[k] = __double2float_rn(si[k] - (double)hi[k]);
    }
    seg[3LL * i] = make_float4(hi[0], hi[1], hi[2], lo[0]);
    seg[3LL * i + 1] = make_float4(lo[1], lo[2], b[0], b[1]);
    seg[3LL * i + 2] = make_float4(b[2], b[0] * b[0] + b[1] * b[1] + b[2] * b[2], 0.f, 0.f);
    // Image of segment i -> q across each solid face: from M(s_q) to M(s_i),
    // M mirroring the normal coordinate x_a -> 2w - x_a (record (1 + f) N + i).
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        if (f >= P.nfaces) break;
        const int code = P.face_code[f], ax = code >> 1;
        const double L = (double)(ax == 0 ? P.g.nx : (ax == 1 ? P.g.ny : P.g.nz));
        const double w2 = 2.0 * ((code & 1) ? L - 0.5 : -0.5);
        float ihi[3], ilo[3], d[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            // a line's last point starts no segment: a zero-length record at its own image
            const double st = q >= 0 ? sq[k] : si[k];
            const double m = k == ax ? w2 - st : st;
            ihi[k] = __double2float_rn(m);
            ilo[k] = __double2float_rn(m - (double)ihi[k]);
            d[k] = k == ax ? b[k] : -b[k];
        }
        const long long r = 3LL * ((long long)(1 + f) * N + i);
        seg[r] = make_float4(ihi[0], ihi[1], ihi[2], ilo[0]);
        seg[r + 1] = make_float4(ilo[1], ilo[2], d[0], d[1]);
        seg[r + 2] = make_float4(d[2], d[0] * d[0] + d[1] * d[1] + d[2] * d[2], 0.f, 0.f);
    }
}

// The equation of motion of each point as a kernel of its own (used when the
// Biot-Savart pass does not apply it).
__global__ void __launch_bounds__(64) k_eom(EomArgs A, const float* __restrict__ vbs) {
    pdl_wait_trigger();
    const int N = A.counters[CNT_N];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < N;
    float v[3] = {0.f, 0.f, 0.f};
    if (valid)
        for (int k = 0; k < 3; ++k) v[k] = vbs[(long long)k * A.cap + i];
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
                           int cap, float4* geo, float4* seg, double* s0_copy, cudaStream_t st) {
    if (cap <= 0) return;
    launch_pdl(k_geometry_stage, (cap + 63) / 64, 64, 0, st, P, s, next, prev, counters, cap, geo, seg, s0_copy);
}

void launch_eom(const EomArgs& A, const float* vbs, cudaStream_t s) {
    if (A.cap <= 0) return;
    launch_pdl(k_eom, (A.cap + 63) / 64, 64, 0, s, A, vbs);
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
