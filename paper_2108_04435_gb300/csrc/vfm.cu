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


// One thread per point (and per padding record position), one block per
// group of BS_GROUP records in point order; thread 0 also resets the work
// counter of the Biot-Savart launch that follows.
__global__ void __launch_bounds__(BS_GROUP) k_geometry_stage(VfmParams P, const double* __restrict__ s,
                                                             const int* __restrict__ next,
                                                             const int* __restrict__ prev,
                                                             int* __restrict__ counters, int cap,
                                                             float4* __restrict__ geo, float4* __restrict__ seg,
                                                             double* __restrict__ s0_copy, BsOrder o) {
    pdl_wait_trigger();
    const int N = counters[CNT_N];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) counters[CNT_BSWORK] = 0;  // the Biot-Savart launch that follows takes items from 0
    bs_point_order_origin(o, s, cap, N);
    __syncthreads();
    if (i >= N) {
        bs_pad_records(N, P.nfaces, i, seg);
        return;
    }
    geometry_point(P, s, next, prev, N, cap, i, geo, seg, s0_copy, o);
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
                           int cap, float4* geo, float4* seg, double* s0_copy, const BsOrder& o, cudaStream_t st) {
    if (cap <= 0) return;
    // padding positions reach the capacity rounded up to a whole group
    const int span = (int)bs_block(cap, 1);
    launch_pdl(k_geometry_stage, span / BS_GROUP, BS_GROUP, 0, st, P, s, next, prev, counters, cap, geo, seg,
               s0_copy, o);
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
