// Nonlocal Biot-Savart velocity of the vortex filaments (Eq. 3 of
// arXiv 2108.04435, integrated segment-wise as Sec. II.A states).
//
// For target r and straight segment s_j -> s_j + d_j, with R1 = s_j - r
// (minimum image on periodic axes) and R2 = R1 + d_j, the exact line integral
// of the Eq. 3 kernel is
//     v = kappa/(4 pi) (R1 x R2) (|R1| + |R2|) / (|R1||R2| (|R1||R2| + R1.R2)).
// The two segments touching the target are left to the local term.
//
// GB300 mapping: one target per thread (position in registers as float hi+lo
// parts, so that R1 keeps ~1e-7 relative accuracy in boxes up to 1024 cells),
// source segments streamed through shared memory in tiles that a single
// thread fetches with TMA bulk copies (cp.async.bulk + mbarrier, double
// buffered), every lane reading each record as a broadcast.  This is FP32 +
// MUFU work (2 rsqrt + 1 reciprocal per pair), not a contraction, so no tensor
// cores.  Small filament sets are split over source chunks (grid.y); the
// partial sums are reduced later in a fixed order.
#include <cuda_runtime.h>
#include <math.h>

#include "vlb_internal.cuh"

namespace vlb {

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for a barrier phase, giving up after ~1 s of clock so that a lost copy
// turns into an error status instead of a hung GPU.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > 2000000000LL) return false;
    }
    return true;
}

struct BoxF {
    float Lx, Ly, Lz, iLx, iLy, iLz;  // 0 on wall axes: no minimum image
};

__device__ __forceinline__ void issue_tile(float4* dst, const float4* seg, int jb, int cnt, uint64_t* bar) {
    const uint32_t bytes = (uint32_t)cnt * 48u;
    mbar_expect_tx(bar, bytes);
    bulk_copy_g2s(dst, seg + 3LL * jb, bytes, bar);
}

template <bool PERIODIC>
__global__ void __launch_bounds__(BS_TPB) k_biot_savart(const float4* __restrict__ seg, const int* __restrict__ prev,
                                                        const int* __restrict__ counters, int cap, BoxF box, float kq,
                                                        float* __restrict__ out, int* __restrict__ status) {
    __shared__ __align__(128) float4 tile[2][BS_TILE * 3];
    __shared__ __align__(8) uint64_t bar[2];
    const int N = counters[CNT_N];
    const int i0 = blockIdx.x * BS_TPB;
    if (i0 >= N) return;
    const int nsplit = gridDim.y, split = blockIdx.y;
    const int chunk = (N + nsplit - 1) / nsplit;
    const int j0 = split * chunk;
    const int j1 = min(N, j0 + chunk);
    const int i = i0 + threadIdx.x;
    const bool valid = i < N;
    float rhx = 0.f, rhy = 0.f, rhz = 0.f, rlx = 0.f, rly = 0.f, rlz = 0.f;
    int self = -1, pi = -1;
    if (valid) {
        const float4 a = seg[3LL * i], b = seg[3LL * i + 1];
        rhx = a.x; rhy = a.y; rhz = a.z; rlx = a.w; rly = b.x; rlz = b.y;
        self = i;
        pi = prev[i];
    }
    float vx = 0.f, vy = 0.f, vz = 0.f;
    const int ntiles = j1 > j0 ? (j1 - j0 + BS_TILE - 1) / BS_TILE : 0;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && ntiles > 0) issue_tile(tile[0], seg, j0, min(BS_TILE, j1 - j0), &bar[0]);
    int consumed = 0;
    bool timed_out = false;
    for (int t = 0; t < ntiles; ++t) {
        const int b = t & 1;
        if (threadIdx.x == 0 && t + 1 < ntiles) {
            const int jn = j0 + (t + 1) * BS_TILE;
            issue_tile(tile[b ^ 1], seg, jn, min(BS_TILE, j1 - jn), &bar[b ^ 1]);
        }
        const bool ok = mbar_wait_bounded(&bar[b], (uint32_t)((t >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        consumed = t + 1;
        const int jb = j0 + t * BS_TILE;
        const int cnt = min(BS_TILE, j1 - jb);
        const float4* T = tile[b];
#pragma unroll 4
        for (int k = 0; k < cnt; ++k) {
            const float4 A = T[3 * k], B = T[3 * k + 1], D = T[3 * k + 2];
            float r1x = (A.x - rhx) + (A.w - rlx);
            float r1y = (A.y - rhy) + (B.x - rly);
            float r1z = (A.z - rhz) + (B.y - rlz);
            if (PERIODIC) {
                r1x -= box.Lx * rintf(r1x * box.iLx);
                r1y -= box.Ly * rintf(r1y * box.iLy);
                r1z -= box.Lz * rintf(r1z * box.iLz);
            }
            const float r2x = r1x + B.z, r2y = r1y + B.w, r2z = r1z + D.x;
            const float a2 = r1x * r1x + r1y * r1y + r1z * r1z;
            const float b2 = r2x * r2x + r2y * r2y + r2z * r2z;
            const float ia = rsqrtf(a2), ib = rsqrtf(b2);
            const float la = a2 * ia, lb = b2 * ib;
            const float ab = la * lb;
            const float dot = r1x * r2x + r1y * r2y + r1z * r2z;
            const float s = ab + dot;
            const float fac = kq * (la + lb) * __frcp_rn(ab * s);
            const int j = jb + k;
            const bool use = (j != self) & (j != pi) & (s > 1e-6f * ab);
            const float c = use ? fac : 0.f;
            vx += c * (r1y * r2z - r1z * r2y);
            vy += c * (r1z * r2x - r1x * r2z);
            vz += c * (r1x * r2y - r1y * r2x);
        }
        __syncthreads();
    }
    if (timed_out) {
        if (threadIdx.x == 0) {
            atomicOr(status, ST_TIMEOUT);
            // let copies still in flight land before the block's shared memory goes away
            for (int t = consumed; t < min(ntiles, consumed + 2); ++t) mbar_wait_bounded(&bar[t & 1], (uint32_t)((t >> 1) & 1));
        }
        return;
    }
    if (valid) {
        out[((long long)split * 3 + 0) * cap + i] = vx;
        out[((long long)split * 3 + 1) * cap + i] = vy;
        out[((long long)split * 3 + 2) * cap + i] = vz;
    }
}

// Stand-alone entry: prev[] and the source records from a caller's point set.
__global__ void k_bs_prep(Grid g, const double* __restrict__ pos, const int* __restrict__ next, int n,
                          int* __restrict__ prev, float4* __restrict__ seg, int* __restrict__ counters) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        counters[CNT_N] = n;
        counters[CNT_STATUS] = 0;
    }
    if (i >= n) return;
    const int q = next[i];
    prev[q] = i;
    const int nn[3] = {g.nx, g.ny, g.nz};
    float hi[3], lo[3], d[3];
    for (int k = 0; k < 3; ++k) {
        const double si = pos[(long long)k * n + i];
        double dd = pos[(long long)k * n + q] - si;
        if (!g.wall[k]) {
            const double L = (double)nn[k];
            if (dd > 0.5 * L) dd -= L;
            else if (dd < -0.5 * L) dd += L;
        }
        hi[k] = __double2float_rn(si);
        lo[k] = __double2float_rn(si - (double)hi[k]);
        d[k] = __double2float_rn(dd);
    }
    seg[3LL * i] = make_float4(hi[0], hi[1], hi[2], lo[0]);
    seg[3LL * i + 1] = make_float4(lo[1], lo[2], d[0], d[1]);
    seg[3LL * i + 2] = make_float4(d[2], 0.f, 0.f, 0.f);
}

__global__ void k_bs_reduce(const float* __restrict__ bsp, int nsplit, int n, int cap, float* __restrict__ vel) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = 0; k < 3; ++k) {
        float s = 0.f;
        for (int m = 0; m < nsplit; ++m) s += bsp[((long long)m * 3 + k) * cap + i];
        vel[(long long)k * n + i] = s;
    }
}

BoxF make_box(const Grid& g) {
    BoxF b;
    b.Lx = g.wall[0] ? 0.f : (float)g.nx;
    b.Ly = g.wall[1] ? 0.f : (float)g.ny;
    b.Lz = g.wall[2] ? 0.f : (float)g.nz;
    b.iLx = g.wall[0] ? 0.f : 1.f / (float)g.nx;
    b.iLy = g.wall[1] ? 0.f : 1.f / (float)g.ny;
    b.iLz = g.wall[2] ? 0.f : 1.f / (float)g.nz;
    return b;
}

}  // namespace

// Source splits for a filament set of about n points: enough blocks to fill
// the GPU (~4 per SM on 152 SMs), with at least 64 segments per split.
int bs_nsplit(int n_hint, int cap) {
    const int n = n_hint > 0 ? n_hint : 1;
    const int tb = (n + BS_TPB - 1) / BS_TPB;
    int ns = (4 * 152 + tb - 1) / tb;
    const int by_chunk = (n + 63) / 64;
    if (ns > by_chunk) ns = by_chunk;
    if (ns < 1) ns = 1;
    if (ns > MAX_SPLIT) ns = MAX_SPLIT;
    (void)cap;
    return ns;
}

void launch_biot_savart(const Grid& g, double kappa, const float4* seg, const int* prev, const int* counters, int cap,
                        int nsplit, float* bsp, cudaStream_t s) {
    if (cap <= 0) return;
    dim3 grid((cap + BS_TPB - 1) / BS_TPB, nsplit);
    const float kq = (float)(kappa / (4.0 * 3.14159265358979323846));
    const BoxF box = make_box(g);
    int* status = const_cast<int*>(counters) + CNT_STATUS;
    if (g.wall[0] && g.wall[1] && g.wall[2])
        k_biot_savart<false><<<grid, BS_TPB, 0, s>>>(seg, prev, counters, cap, box, kq, bsp, status);
    else
        k_biot_savart<true><<<grid, BS_TPB, 0, s>>>(seg, prev, counters, cap, box, kq, bsp, status);
}

void launch_bs_standalone_prep(const Grid& g, const double* pos, const int* next, int n, int* prev, float4* seg,
                               int* counters, cudaStream_t s) {
    k_bs_prep<<<(n + 255) / 256 > 0 ? (n + 255) / 256 : 1, 256, 0, s>>>(g, pos, next, n, prev, seg, counters);
}

void launch_bs_reduce(const float* bsp, int nsplit, int n, int cap, float* vel, cudaStream_t s) {
    if (n <= 0) return;
    k_bs_reduce<<<(n + 255) / 256, 256, 0, s>>>(bsp, nsplit, n, cap, vel);
}

}  // namespace vlb
