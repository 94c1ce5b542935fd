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

#include <mutex>

#include "eom.cuh"
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

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Nearest integer of x * inv (|x * inv| < 2^22) on the FMA pipe, in two
// instructions: adding 1.5 * 2^23 to the exact product rounds it to the
// nearest integer in FP32, and removing it again is exact.
__device__ __forceinline__ float round_mul_fma(float x, float inv) {
    const float M = 12582912.0f;
    return __fsub_rn(__fmaf_rn(x, inv, M), M);
}

__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// One target of a Biot-Savart tile pass (registers of one thread).
struct BsTarget {
    float hx, hy, hz, lx, ly, lz;  // position, float hi + lo parts
    float vx, vy, vz;              // accumulated velocity
    int self, prev;                // its own segment and its predecessor's (local term)
    int excl;                      // a pinned end: the image of its own segment across its wall (local term)
};

// One (target, segment) pair of Eq. 3.  With R1 = s_j - r and d the segment
// vector: R1 x R2 = R1 x d, R1.R2 = |R1|^2 + R1.d and |R2|^2 = |R1|^2 +
// 2 R1.d + |d|^2 (|d|^2 stored in the record).  MASKED: j may be the target's
// own segment or its predecessor's, which belong to the local term.
template <bool PERIODIC, bool MASKED>
__device__ __forceinline__ void bs_pair(const float4& A, const float4& B, const float4& D, int j, BsTarget& t,
                                        const BoxF& box, float kq) {
    const float dx = B.z, dy = B.w, dz = D.x, dd = D.y;
    float r1x = (A.x - t.hx) + (A.w - t.lx);
    float r1y = (A.y - t.hy) + (B.x - t.ly);
    float r1z = (A.z - t.hz) + (B.y - t.lz);
    if (PERIODIC) {
        r1x = fmaf(-box.Lx, round_mul_fma(r1x, box.iLx), r1x);
        r1y = fmaf(-box.Ly, round_mul_fma(r1y, box.iLy), r1y);
        r1z = fmaf(-box.Lz, round_mul_fma(r1z, box.iLz), r1z);
    }
    const float a2 = r1x * r1x + r1y * r1y + r1z * r1z;
    const float rd = r1x * dx + r1y * dy + r1z * dz;
    const float b2 = fmaf(2.f, rd, a2) + dd;
    const float ia = rsqrt_approx(a2), ib = rsqrt_approx(b2);
    const float la = a2 * ia, lb = b2 * ib;
    const float ab = la * lb;
    const float s = ab + (a2 + rd);
    const float fac = kq * (la + lb) * rcp_approx(ab * s);
    // s <= 1e-6 ab: the target lies on the segment (or coincides with an
    // end point), where the integral is not defined; NaN fails the test too
    bool use = s > 1e-6f * ab;
    if (MASKED) use = use & (j != t.self) & (j != t.prev) & (j != t.excl);
    const float c = use ? fac : 0.f;
    t.vx += c * (r1y * dz - r1z * dy);
    t.vy += c * (r1z * dx - r1x * dz);
    t.vz += c * (r1x * dy - r1y * dx);
}

// Sum over the segments of one shared-memory tile for TGT targets per thread.
// Four segments per unrolled pass: with few points a block's four warps are
// alone on their SM, and the pair arithmetic is a chain of dependent
// instructions (measured: 1.2% faster coupled step at 1.1k points, 0.6% at
// 17k, than two per pass).
template <bool PERIODIC, bool MASKED, int TGT>
__device__ __forceinline__ void bs_tile(const float4* __restrict__ T, int cnt, int jb, BsTarget (&t)[TGT],
                                        const BoxF& box, float kq) {
#pragma unroll 4
    for (int k = 0; k < cnt; ++k) {
        const float4 A = T[3 * k], B = T[3 * k + 1], D = T[3 * k + 2];
#pragma unroll
        for (int u = 0; u < TGT; ++u) bs_pair<PERIODIC, MASKED>(A, B, D, jb + k, t[u], box, kq);
    }
}

// Work items are (target tile of BS_TPB points, source split).  Block b
// starts with item b and takes further items from a device counter (reset by
// the stage-geometry kernel), so the grid is fixed and no item depends on a
// host-side estimate of N.  With several splits, each item stores its partial
// sums and the last item of a target tile adds them in split order (fixed,
// hence deterministic) into vel; with one split the item writes vel directly.
struct BsImages {
    int nfaces;
    int face_code[6];
    const float4* geo;  // pinned-end wall codes (+1) in geo[2i + 1].w
};

// Target i of N (none when i >= N): its position from its own segment record,
// and the segments that belong to its local term.
__device__ __forceinline__ BsTarget bs_target(const float4* __restrict__ seg, const int* __restrict__ prev,
                                              const BsImages& im, int N, int i) {
    BsTarget t{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, -1, -1, -1};
    if (i < N) {
        const float4 a = seg[3LL * i], b = seg[3LL * i + 1];
        t.hx = a.x; t.hy = a.y; t.hz = a.z; t.lx = a.w; t.ly = b.x; t.lz = b.y;
        t.self = i;
        t.prev = prev[i];
        if (im.nfaces > 0) {
            const int pin = (int)im.geo[2LL * i + 1].w - 1;
#pragma unroll
            for (int f = 0; f < 6; ++f)
                if (f < im.nfaces && im.face_code[f] == pin) t.excl = (1 + f) * N + (t.prev < 0 ? i : t.prev);
        }
    }
    return t;
}

// Shared memory of one block's Biot-Savart work: two source tiles, their
// mbarriers and two broadcast slots.  `used` counts the tiles the block has
// consumed (buffer = used & 1, phase = (used >> 1) & 1) across calls.
struct BsSmem {
    float4 (*tile)[BS_TILE * 3];
    uint64_t* bar;
    int* s_item;
    int* s_last;
};

__device__ __forceinline__ void bs_smem_init(const BsSmem& sm) {
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
    }
}

// The work items of one Biot-Savart pass taken by this block: the item
// blockIdx.x, then items from the device counter CNT_BSWORK (reset to 0
// before the pass).  Returns false after a timed-out tile copy (status
// TIMEOUT set).
template <bool PERIODIC, int TGT, bool EOM, bool ACC>
__device__ bool bs_work(const float4* __restrict__ seg, const int* __restrict__ prev, int* __restrict__ counters,
                        int* __restrict__ tile_ticket, int cap, const BoxF& box, float kq, float* __restrict__ part,
                        float* __restrict__ vel, const EomArgs& ea, const BsImages& im, const BsSmem& sm,
                        uint32_t& used, long long* __restrict__ vacc) {
    float4 (*tile)[BS_TILE * 3] = sm.tile;
    uint64_t* bar = sm.bar;
    int& s_item = *sm.s_item;
    int& s_last = *sm.s_last;
    constexpr int TT = BS_TPB * TGT;  // targets per item
    const int N = counters[CNT_N];
    if (N <= 0) return true;
    const int ns = bs_splits(N, TT);
    const int ntb = (N + TT - 1) / TT;
    const int nitems = ntb * ns;
    const int nsrc = N * (1 + im.nfaces);  // segments, then their wall images
    const int chunk = (nsrc + ns - 1) / ns;
    if ((int)blockIdx.x >= nitems) return true;
    int item = blockIdx.x;
    while (true) {
        __syncthreads();
        const int tb = item % ntb, split = item / ntb;
        const int j0 = split * chunk;
        const int j1 = min(nsrc, j0 + chunk);
        BsTarget t[TGT];
        bool own_any = false;
#pragma unroll
        for (int u = 0; u < TGT; ++u) t[u] = bs_target(seg, prev, im, N, tb * TT + u * BS_TPB + threadIdx.x);
        const int ntiles = j1 > j0 ? (j1 - j0 + BS_TILE - 1) / BS_TILE : 0;
        if (threadIdx.x == 0 && ntiles > 0) issue_tile(tile[used & 1], seg, j0, min(BS_TILE, j1 - j0), &bar[used & 1]);
        for (int tt = 0; tt < ntiles; ++tt) {
            const uint32_t u = used + (uint32_t)tt;
            const int b = (int)(u & 1u);
            if (threadIdx.x == 0 && tt + 1 < ntiles) {
                const int jn = j0 + (tt + 1) * BS_TILE;
                issue_tile(tile[b ^ 1], seg, jn, min(BS_TILE, j1 - jn), &bar[b ^ 1]);
            }
            const bool ok = mbar_wait_bounded(&bar[b], (u >> 1) & 1u);
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) {
                    atomicOr(&counters[CNT_STATUS], ST_TIMEOUT);
                    // let a copy still in flight land before the block's shared memory goes away
                    if (tt + 1 < ntiles) mbar_wait_bounded(&bar[b ^ 1], ((u + 1u) >> 1) & 1u);
                }
                return false;
            }
            const int jb = j0 + tt * BS_TILE;
            const int cnt = min(BS_TILE, j1 - jb);
            own_any = false;
#pragma unroll
            for (int v = 0; v < TGT; ++v)
                own_any |= (unsigned)(t[v].self - jb) < (unsigned)cnt || (unsigned)(t[v].prev - jb) < (unsigned)cnt ||
                           (unsigned)(t[v].excl - jb) < (unsigned)cnt;
            if (__any_sync(0xffffffffu, own_any))
                bs_tile<PERIODIC, true, TGT>(tile[b], cnt, jb, t, box, kq);
            else
                bs_tile<PERIODIC, false, TGT>(tile[b], cnt, jb, t, box, kq);
            __syncthreads();
        }
        used += (uint32_t)ntiles;
        if (ACC) {
            // ACC: each split adds its sums in fixed point (exact, in any
            // order); the equation-of-motion kernel that follows reads them
#pragma unroll
            for (int v = 0; v < TGT; ++v) {
                const int i = t[v].self;
                if (i >= 0) {
                    atomicAdd((unsigned long long*)&vacc[i], (unsigned long long)bs_fixed(t[v].vx));
                    atomicAdd((unsigned long long*)&vacc[(long long)cap + i], (unsigned long long)bs_fixed(t[v].vy));
                    atomicAdd((unsigned long long*)&vacc[2LL * cap + i], (unsigned long long)bs_fixed(t[v].vz));
                }
            }
        } else if (ns == 1) {
#pragma unroll
            for (int v = 0; v < TGT; ++v) {
                const int i = t[v].self;
                if (EOM) {
                    eom_point(ea, i, i >= 0, t[v].vx, t[v].vy, t[v].vz);
                } else if (i >= 0) {
                    vel[i] = t[v].vx;
                    vel[(long long)cap + i] = t[v].vy;
                    vel[2LL * cap + i] = t[v].vz;
                }
            }
        } else {
#pragma unroll
            for (int v = 0; v < TGT; ++v) {
                const int i = t[v].self;
                if (i >= 0) {
                    part[((long long)split * 3 + 0) * cap + i] = t[v].vx;
                    part[((long long)split * 3 + 1) * cap + i] = t[v].vy;
                    part[((long long)split * 3 + 2) * cap + i] = t[v].vz;
                }
            }
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) s_last = atomicAdd(&tile_ticket[tb], 1) == ns - 1;
            __syncthreads();
            if (s_last) {
                __threadfence();
#pragma unroll
                for (int v = 0; v < TGT; ++v) {
                    const int i = t[v].self;
                    float a[3] = {0.f, 0.f, 0.f};
                    if (i >= 0) {
                        for (int m = 0; m < ns; ++m)
#pragma unroll
                            for (int k = 0; k < 3; ++k) a[k] += __ldcg(&part[((long long)m * 3 + k) * cap + i]);
                    }
                    if (EOM) {
                        eom_point(ea, i, i >= 0, a[0], a[1], a[2]);
                    } else if (i >= 0) {
                        vel[i] = a[0];
                        vel[(long long)cap + i] = a[1];
                        vel[2LL * cap + i] = a[2];
                    }
                }
                if (threadIdx.x == 0) tile_ticket[tb] = 0;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_item = (int)gridDim.x + atomicAdd(&counters[CNT_BSWORK], 1);
        __syncthreads();
        item = s_item;
        if (item >= nitems) break;
    }
    return true;
}

// At least 8 resident blocks of 128 threads per SM (the grid is sized for 8):
// the pair loop is issue-bound and needs the warps, and the equation of motion
// applied after it (EOM) would otherwise raise the count to 72 registers.
template <bool PERIODIC, int TGT, bool EOM, bool ACC>
__global__ void __launch_bounds__(BS_TPB, EOM ? 8 : 9)
    k_biot_savart(const float4* __restrict__ seg, const int* __restrict__ prev, int* __restrict__ counters,
                  int* __restrict__ tile_ticket, int cap, BoxF box, float kq, float* __restrict__ part,
                  float* __restrict__ vel, EomArgs ea, BsImages im, long long* __restrict__ vacc) {
    pdl_wait_trigger();
    __shared__ __align__(128) float4 tile[2][BS_TILE * 3];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_item, s_last;
    const BsSmem sm = {tile, bar, &s_item, &s_last};
    bs_smem_init(sm);
    uint32_t used = 0;
    bs_work<PERIODIC, TGT, EOM, ACC>(seg, prev, counters, tile_ticket, cap, box, kq, part, vel, ea, im, sm, used,
                                     vacc);
}

// Stand-alone entry: prev[] and the source records from a caller's point set.
__global__ void k_bs_prep(Grid g, const double* __restrict__ pos, const int* __restrict__ next, int n,
                          int* __restrict__ prev, float4* __restrict__ seg, int* __restrict__ counters) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        counters[CNT_N] = n;
        counters[CNT_STATUS] = 0;
        counters[CNT_BSWORK] = 0;
    }
    if (i >= n) return;
    int q = next[i];
    if (q < -1 || q >= n) {  // not a point index: no segment
        atomicOr(&counters[CNT_STATUS], ST_TOPOLOGY);
        q = -1;
    }
    if (q >= 0) prev[q] = i;
    const int nn[3] = {g.nx, g.ny, g.nz};
    float hi[3], lo[3], d[3];
    for (int k = 0; k < 3; ++k) {
        const double si = pos[(long long)k * n + i];
        double dd = q >= 0 ? pos[(long long)k * n + q] - si : 0.0;
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
    seg[3LL * i + 2] = make_float4(d[2], d[0] * d[0] + d[1] * d[1] + d[2] * d[2], 0.f, 0.f);
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

// Up to BS_ACC_MAX points the split sums go to the fixed-point accumulator,
// so no block waits for a ticket and no last block re-reads partial sums.
bool bs_uses_vacc(int n_hint) { return n_hint < BS_ACC_MAX; }

int bs_max_splits(int cap) {
    int m = 1;
    for (int n = 1; n <= cap; n += (n < 8192 ? 1 : 128)) {
        const int k = bs_splits(n, BS_TPB);
        if (k > m) m = k;
    }
    return m;
}

template <int TGT, bool EOM, bool ACC = false>
void bs_launch(const Grid& g, float kq, const float4* seg, const int* prev, int* cnt, int* tile_ticket, int cap, int n,
               float* part, float* vel, const EomArgs& ea, const BsImages& im, cudaStream_t s,
               long long* vacc = nullptr) {
    // enough blocks for every item of about n points (at most 8 per SM); more
    // points than that are still covered by the blocks' item loop
    constexpr int TT = BS_TPB * TGT;
    const int items = ((n + TT - 1) / TT) * bs_splits(n, TT);
    const int grid = items < 8 * 152 ? items : 8 * 152;
    const BoxF box = make_box(g);
    if (g.wall[0] && g.wall[1] && g.wall[2])
        launch_pdl(k_biot_savart<false, TGT, EOM, ACC>, grid, BS_TPB, 0, s, seg, prev, cnt, tile_ticket, cap, box, kq,
                   part, vel, ea, im, vacc);
    else
        launch_pdl(k_biot_savart<true, TGT, EOM, ACC>, grid, BS_TPB, 0, s, seg, prev, cnt, tile_ticket, cap, box, kq,
                   part, vel, ea, im, vacc);
}

void launch_biot_savart(const Grid& g, double kappa, const float4* seg, const int* prev, const int* counters,
                        int* tile_ticket, int cap, int n_hint, float* part, float* vel, cudaStream_t s,
                        const EomArgs* eom, int nfaces, const int* face_code, const float4* geo,
                        long long* vacc) {
    if (cap <= 0) return;
    const int n = n_hint > 0 ? (n_hint < cap ? n_hint : cap) : 1;
    const float kq = (float)(kappa / (4.0 * 3.14159265358979323846));
    int* cnt = const_cast<int*>(counters);
    // two targets per thread from 8192 points on (each shared-memory record is
    // then read once for both; 1% faster at 17k points, the same at 86k)
    const EomArgs none = {};
    const EomArgs& ea = eom ? *eom : none;
    BsImages im = {};
    im.nfaces = geo ? nfaces : 0;
    for (int f = 0; f < im.nfaces; ++f) im.face_code[f] = face_code[f];
    im.geo = geo;
    if (vacc && !eom && bs_uses_vacc(n)) {
        if (n >= 8192) bs_launch<2, false, true>(g, kq, seg, prev, cnt, tile_ticket, cap, n, part, vel, ea, im, s, vacc);
        else bs_launch<1, false, true>(g, kq, seg, prev, cnt, tile_ticket, cap, n, part, vel, ea, im, s, vacc);
        return;
    }
    if (n >= 8192) {
        if (eom) bs_launch<2, true>(g, kq, seg, prev, cnt, tile_ticket, cap, n, part, vel, ea, im, s);
        else bs_launch<2, false>(g, kq, seg, prev, cnt, tile_ticket, cap, n, part, vel, ea, im, s);
    } else {
        if (eom) bs_launch<1, true>(g, kq, seg, prev, cnt, tile_ticket, cap, n, part, vel, ea, im, s);
        else bs_launch<1, false>(g, kq, seg, prev, cnt, tile_ticket, cap, n, part, vel, ea, im, s);
    }
}

void launch_bs_standalone_prep(const Grid& g, const double* pos, const int* next, int n, int* prev, float4* seg,
                               int* counters, cudaStream_t s) {
    cudaMemsetAsync(prev, 0xff, sizeof(int) * (size_t)n, s);  // first points of open lines keep -1
    k_bs_prep<<<(n + 255) / 256 > 0 ? (n + 255) / 256 : 1, 256, 0, s>>>(g, pos, next, n, prev, seg, counters);
}

}  // namespace vlb

// ---------------------------------------------------------------------------
// Allocation-free variant of the stand-alone Biot-Savart entry point, for
// callers that may not allocate device memory while they run (for example a
// host framework that only hands out pre-registered buffers, or code running
// where cudaMalloc would synchronise the device).  Its scratch space is a
// file-scope device array of fixed size that every GPU loading this library
// holds until the process exits.

namespace {

constexpr int NOALLOC_MAX_POINTS = 65536;
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(6) << 20;  // >= vlb_biot_savart_scratch_bytes(65536)
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_bs_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_bs_scratch_mu;
void* g_bs_scratch_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of g_bs_scratch on the current device.  In host code the
// name g_bs_scratch is only a host-side stand-in, so the address is asked
// from the runtime once per device (with that device current) and cached.
int noalloc_scratch(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        cudaGetLastError();
        return vlb::set_error(VLB_ERR_CUDA, "no usable current CUDA device");
    }
    std::lock_guard<std::mutex> lock(g_bs_scratch_mu);
    if (!g_bs_scratch_addr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_bs_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return vlb::set_error(VLB_ERR_CUDA, "cudaGetSymbolAddress of the Biot-Savart scratch failed");
        }
        g_bs_scratch_addr[dev] = ptr;
    }
    *out = g_bs_scratch_addr[dev];
    return VLB_OK;
}

}  // namespace

extern "C" int vlb_biot_savart_noalloc(const vlb_params* p, const double* pos, const int32_t* next, int32_t n,
                                       float* vel, void* stream) {
    if (n > NOALLOC_MAX_POINTS)
        return vlb::set_error(VLB_ERR_INVALID_ARG,
                              "vlb_biot_savart_noalloc: n exceeds its 65536-point limit (use vlb_biot_savart)");
    if (vlb_biot_savart_scratch_bytes(n) > NOALLOC_SCRATCH_BYTES)
        return vlb::set_error(VLB_ERR_INVALID_ARG, "vlb_biot_savart_noalloc: scratch array too small");
    void* scratch = nullptr;
    const int rc = noalloc_scratch(&scratch);
    if (rc != VLB_OK) return rc;
    return vlb::bs_standalone(p, pos, next, n, vel, scratch, NOALLOC_SCRATCH_BYTES, stream);
}
