// Spatial order of the Biot-Savart sources (the points of the current step):
// a Morton key per point from its bin of 16 cells (wider on lattices of more
// than 65536 bins), a counting sort over the bins, and inside each bin the
// points in ascending index, so that the order depends on nothing but the
// positions (and a line's points, numbered along it, mostly stay
// consecutive).  Built once per step from BS_SORT_MIN points on.
//
// Then, in any order, the source slots: every sorted position k takes slot
// k + (gap slots before it), a gap slot following k when the successor of
// its point is not the point at k + 1; a two-kernel scan (gap counts per
// block, then each block's prefix from the counts before it), which also
// records what every slot holds.  Group g of BS_GROUP slots gets the integer
// origin of its first slot's point.
#include <cuda_runtime.h>
#include <math.h>

#include "vlb_internal.cuh"

namespace vlb {

namespace {

__device__ __forceinline__ int bs_key_of(const Grid& g, const BsBins& bb, double x, double y, double z) {
    const int n[3] = {g.nx, g.ny, g.nz};
    const double s[3] = {x, y, z};
    int b[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int c = (int)floor(s[a]);
        c = c < 0 ? 0 : (c > n[a] - 1 ? n[a] - 1 : c);
        b[a] = c >> bb.shift;
    }
    int key = 0, pos = 0;
    for (int l = 0; l < 16; ++l)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (l < bb.bits[a]) key |= ((b[a] >> l) & 1) << pos++;
    return key;
}

// Key and bin count of every point (grid-stride beyond the grid).
__global__ void k_sort_keys(Grid g, BsBins bb, const double* __restrict__ pos, int cap,
                            const int* __restrict__ counters, int* __restrict__ key, int* __restrict__ cnt) {
    pdl_wait_trigger();
    const int N = counters[CNT_N];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const int k = bs_key_of(g, bb, pos[i], pos[(long long)cap + i], pos[2LL * cap + i]);
        key[i] = k;
        atomicAdd(&cnt[k], 1);
    }
}

// Exclusive scan of the bin counts (one block of 1024 threads), 4096 bins
// per round: each thread takes four consecutive bins with one 16-byte load
// (a warp reads 512 contiguous bytes), the block scans the thread sums, and
// a carry runs from round to round.  K is a power of two.
__global__ void __launch_bounds__(1024) k_sort_scan(int K, const int* __restrict__ cnt, int* __restrict__ start) {
    pdl_wait_trigger();
    __shared__ int warp_sum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int carry = 0;
    for (int base = 0; base < K; base += 4096) {
        const int k0 = base + 4 * (int)threadIdx.x;
        int4 v = make_int4(0, 0, 0, 0);
        if (k0 + 3 < K) {
            v = *reinterpret_cast<const int4*>(cnt + k0);
        } else if (k0 < K) {
            v.x = cnt[k0];
            if (k0 + 1 < K) v.y = cnt[k0 + 1];
            if (k0 + 2 < K) v.z = cnt[k0 + 2];
        }
        const int sum = v.x + v.y + v.z + v.w;
        int x = sum;  // inclusive scan within the warp
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) warp_sum[w] = x;
        __syncthreads();
        if (w == 0) {
            int z = warp_sum[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, z, off);
                if (lane >= off) z += y;
            }
            warp_sum[lane] = z;  // inclusive over warps
        }
        __syncthreads();
        const int excl = carry + (x - sum) + (w > 0 ? warp_sum[w - 1] : 0);
        if (k0 + 3 < K) {
            *reinterpret_cast<int4*>(start + k0) = make_int4(excl, excl + v.x, excl + v.x + v.y, excl + v.x + v.y + v.z);
        } else if (k0 < K) {
            start[k0] = excl;
            if (k0 + 1 < K) start[k0 + 1] = excl + v.x;
            if (k0 + 2 < K) start[k0 + 2] = excl + v.x + v.y;
        }
        carry += warp_sum[31];
        __syncthreads();  // warp_sum is rewritten by the next round
    }
}

// Every point into its bin (arbitrary order inside the bin; start[k] ends as
// the bin's end).
__global__ void k_sort_scatter(const int* __restrict__ counters, const int* __restrict__ key, int* __restrict__ start,
                               int* __restrict__ tmp) {
    pdl_wait_trigger();
    const int N = counters[CNT_N];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        tmp[atomicAdd(&start[key[i]], 1)] = i;
}

// One warp per bin: the bin's points in ascending index (so the order is
// deterministic), their ranks, and the bin count cleared for the next sort.
__global__ void k_sort_bins(int K, int* __restrict__ cnt, const int* __restrict__ start, const int* __restrict__ tmp,
                            int* __restrict__ ord, int* __restrict__ rank) {
    pdl_wait_trigger();
    const int lane = threadIdx.x & 31;
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= K) return;
    const int n = cnt[k];
    if (n == 0) return;
    const int e = start[k], s0 = e - n;
    for (int c = 0; c < n; c += 32) {
        const int my = c + lane < n ? tmp[s0 + c + lane] : 0x7fffffff;
        int r = 0;
        for (int m = 0; m < n; m += 32) {
            const int other = m + lane < n ? tmp[s0 + m + lane] : 0x7fffffff;
#pragma unroll 8
            for (int q = 0; q < 32; ++q) r += __shfl_sync(0xffffffffu, other, q) < my;
        }
        if (c + lane < n) {
            const int p = s0 + r;
            ord[p] = my;
            rank[my] = p;
        }
    }
    __syncwarp();
    if (lane == 0) cnt[k] = 0;
}

__device__ __forceinline__ int bs_point_at(const BsOrder& o, int k) { return o.sorted ? o.ord[k] : k; }

// 1 when sorted position k needs a gap slot after its own: its point has a
// successor (an index outside [0, N) counts as none) that is not the point
// at k + 1.
__device__ __forceinline__ int bs_gap_after(const BsOrder& o, const int* __restrict__ next, int N, int k) {
    const int q = next[bs_point_at(o, k)];
    if (q < 0 || q >= N) return 0;
    return (k + 1 >= N || bs_point_at(o, k + 1) != q) ? 1 : 0;
}

// Sum of v over the block (1024 threads); every thread gets it.
__device__ __forceinline__ int block_sum_1024(int v, int* warp_sum) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) warp_sum[w] = v;
    __syncthreads();
    int t = warp_sum[lane];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    __syncthreads();  // warp_sum may be rewritten next
    return t;
}

// The contiguous range of sorted positions of this block.
__device__ __forceinline__ void slot_range(int N, int& k0, int& k1) {
    const int ch = (N + (int)gridDim.x - 1) / (int)gridDim.x;
    k0 = min(N, (int)blockIdx.x * ch);
    k1 = min(N, k0 + ch);
}

__global__ void __launch_bounds__(1024) k_slot_count(const int* __restrict__ next, const int* __restrict__ counters,
                                                     BsOrder o, int* __restrict__ bsum) {
    pdl_wait_trigger();
    __shared__ int warp_sum[32];
    const int N = counters[CNT_N];
    int k0, k1;
    slot_range(N, k0, k1);
    int c = 0;
    for (int k = k0 + (int)threadIdx.x; k < k1; k += blockDim.x) c += bs_gap_after(o, next, N, k);
    c = block_sum_1024(c, warp_sum);
    if (threadIdx.x == 0) bsum[blockIdx.x] = c;
}

__device__ __forceinline__ int4 cell_of(const double* __restrict__ pos, int cap, int i) {
    return make_int4((int)floor(pos[i]), (int)floor(pos[(long long)cap + i]), (int)floor(pos[2LL * cap + i]), 0);
}

__global__ void __launch_bounds__(1024) k_slot_assign(const double* __restrict__ pos, const int* __restrict__ next,
                                                      int cap, int* __restrict__ counters, BsOrder o,
                                                      const int* __restrict__ bsum) {
    pdl_wait_trigger();
    __shared__ int warp_sum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int N = counters[CNT_N];
    int k0, k1;
    slot_range(N, k0, k1);
    int pre = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += blockDim.x) pre += bsum[b];
    int carry = block_sum_1024(pre, warp_sum);
    int* slot = const_cast<int*>(o.slot);
    for (int base = k0; base < k1; base += blockDim.x) {
        const int k = base + (int)threadIdx.x;
        const int gap = k < k1 ? bs_gap_after(o, next, N, k) : 0;
        int x = gap;  // inclusive scan within the warp
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) warp_sum[w] = x;
        __syncthreads();
        if (w == 0) {
            int z = warp_sum[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, z, off);
                if (lane >= off) z += y;
            }
            warp_sum[lane] = z;  // inclusive over warps
        }
        __syncthreads();
        if (k < k1) {
            const int sl = k + carry + (x - gap) + (w > 0 ? warp_sum[w - 1] : 0);
            slot[k] = sl;
            const int i = bs_point_at(o, k);
            o.pt[sl] = i;
            if (gap) o.pt[sl + 1] = -2 - i;
            if (sl % BS_GROUP == 0) o.org[sl / BS_GROUP] = cell_of(pos, cap, i);
            if (gap && (sl + 1) % BS_GROUP == 0) o.org[(sl + 1) / BS_GROUP] = cell_of(pos, cap, next[i]);
        }
        carry += warp_sum[31];
        __syncthreads();  // warp_sum is rewritten by the next round
    }
    if (blockIdx.x != gridDim.x - 1) return;
    // the last block: the slot count, padding up to a whole group
    const int ns = N + carry;
    if (threadIdx.x == 0) counters[CNT_NSLOT] = ns;
    const int npad = (int)(bs_block(ns) - ns);
    if ((int)threadIdx.x < npad) o.pt[ns + threadIdx.x] = -1;
}

}  // namespace

void launch_bs_sort(const Grid& g, const double* pos, int cap, int span, const int* counters, int* key, int* tmp,
                    int* ord, int* rank, int* cnt, int* start, cudaStream_t s) {
    const BsBins bb = bs_bins(g.nx, g.ny, g.nz);
    const int blocks = (span + 255) / 256 > 0 ? (span + 255) / 256 : 1;
    launch_pdl(k_sort_keys, blocks, 256, 0, s, g, bb, pos, cap, counters, key, cnt);
    launch_pdl(k_sort_scan, 1, 1024, 0, s, bb.K, (const int*)cnt, start);
    launch_pdl(k_sort_scatter, blocks, 256, 0, s, counters, (const int*)key, start, tmp);
    launch_pdl(k_sort_bins, (bb.K * 32 + 255) / 256, 256, 0, s, bb.K, cnt, (const int*)start, (const int*)tmp, ord,
               rank);
}

void launch_bs_slots(const double* pos, const int* next, int cap, int span, int* counters, const BsOrder& o,
                     int* bsum, cudaStream_t s) {
    int blocks = (span + 1023) / 1024;
    blocks = blocks < 1 ? 1 : (blocks > BS_SLOT_BLOCKS ? BS_SLOT_BLOCKS : blocks);
    launch_pdl(k_slot_count, blocks, 1024, 0, s, next, (const int*)counters, o, bsum);
    launch_pdl(k_slot_assign, blocks, 1024, 0, s, pos, next, cap, counters, o, (const int*)bsum);
}

}  // namespace vlb
