// Spatial order of the Biot-Savart sources (the points of the current step):
// a Morton key per point from its bin (16 cells wide or more, see bs_bins),
// a stable counting sort over the bins, so that inside each bin the points
// keep ascending index and the order depends on nothing but the positions
// (and a line's points, numbered along it, mostly stay consecutive).  Built
// once per step from BS_SORT_MIN points on.
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

// The sort is a stable counting sort over the bins (a key has at most 8
// bits, see bs_bins), in three launches over blocks of SORT_BLOCK
// consecutive point indices: each block counts its points per bin; one block
// scans the counts bin-major (bin 0 of every block, then bin 1, ...); each
// block then places its points, a point's place being the scanned count of
// its bin and block plus the points of its bin before it in the block (by
// warp, then by lane).  Inside a bin the points so keep ascending index, and
// the order depends on the positions alone.  No atomic touches global memory
// (few wide bins would make atomic counters a hot spot) and no step
// compares the points of a bin with each other (a wide bin can hold
// thousands).
constexpr int SORT_BLOCK = 1024;

// Key of every point of block b, and the block's count per bin at
// hist[key * nblk + b] (keys K and beyond: zero).
__global__ void __launch_bounds__(SORT_BLOCK) k_sort_count(Grid g, BsBins bb, const double* __restrict__ pos, int cap,
                                                           const int* __restrict__ counters, int* __restrict__ key,
                                                           int* __restrict__ hist, int nblk) {
    pdl_wait_trigger();
    __shared__ int h[256];
    const int N = counters[CNT_N];
    const int i = blockIdx.x * SORT_BLOCK + threadIdx.x;
    if (threadIdx.x < 256) h[threadIdx.x] = 0;
    __syncthreads();
    if (i < N) {
        const int k = bs_key_of(g, bb, pos[i], pos[(long long)cap + i], pos[2LL * cap + i]);
        key[i] = k;
        atomicAdd(&h[k], 1);
    }
    __syncthreads();
    if ((int)threadIdx.x < bb.K) hist[threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan in place of L counts (one block of 1024 threads), 4096 per
// round: each thread takes four consecutive counts with one 16-byte load
// (a warp reads 512 contiguous bytes), the block scans the thread sums, and
// a carry runs from round to round.  Every thread writes back only the
// counts it read, so the scan can run in place.
__global__ void __launch_bounds__(1024) k_sort_scan(int L, int* v) {
    pdl_wait_trigger();
    __shared__ int warp_sum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int carry = 0;
    for (int base = 0; base < L; base += 4096) {
        const int k0 = base + 4 * (int)threadIdx.x;
        int4 c = make_int4(0, 0, 0, 0);
        if (k0 + 3 < L) {
            c = *reinterpret_cast<const int4*>(v + k0);
        } else if (k0 < L) {
            c.x = v[k0];
            if (k0 + 1 < L) c.y = v[k0 + 1];
            if (k0 + 2 < L) c.z = v[k0 + 2];
        }
        const int sum = c.x + c.y + c.z + c.w;
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
        if (k0 + 3 < L) {
            *reinterpret_cast<int4*>(v + k0) = make_int4(excl, excl + c.x, excl + c.x + c.y, excl + c.x + c.y + c.z);
        } else if (k0 < L) {
            v[k0] = excl;
            if (k0 + 1 < L) v[k0 + 1] = excl + c.x;
            if (k0 + 2 < L) v[k0 + 2] = excl + c.x + c.y;
        }
        carry += warp_sum[31];
        __syncthreads();  // warp_sum is rewritten by the next round
    }
}

// Place of every point of block b: the scanned count of its bin and block,
// plus its rank among the points of its bin in the warps before its own
// (per-warp counts in shared memory, summed over the warps per bin), plus
// its rank among the lanes of its warp with the same bin (a match over the
// warp).  Writes ord (point at each sorted position) and rank (sorted
// position of each point).
__global__ void __launch_bounds__(SORT_BLOCK) k_sort_place(int K, const int* __restrict__ counters,
                                                           const int* __restrict__ key, const int* __restrict__ hist,
                                                           int nblk, int* __restrict__ ord, int* __restrict__ rank) {
    pdl_wait_trigger();
    constexpr int NW = SORT_BLOCK / 32;
    __shared__ int wc[NW][256];
    const int N = counters[CNT_N];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * SORT_BLOCK + threadIdx.x;
    const bool live = i < N;
    const int k = live ? key[i] : K;  // dead lanes match only each other
    for (int e = threadIdx.x; e < NW * 256; e += SORT_BLOCK) (&wc[0][0])[e] = 0;
    const unsigned peers = __match_any_sync(0xffffffffu, k);
    const int before = __popc(peers & ((1u << lane) - 1u));
    __syncthreads();
    if (live && before == 0) wc[w][k] = __popc(peers);
    __syncthreads();
    if ((int)threadIdx.x < K) {
        int run = 0;
        for (int u = 0; u < NW; ++u) {
            const int c = wc[u][threadIdx.x];
            wc[u][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
    if (live) {
        const int p = hist[k * nblk + blockIdx.x] + wc[w][k] + before;
        ord[p] = i;
        rank[i] = p;
    }
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

// hist holds cap ints.  The counts take K * nblk of them, at most
// 256 * ceil(cap / 1024) <= cap / 4 + 256, which is below cap from 342
// points on; both callers sort only from BS_SORT_MIN points on.
void launch_bs_sort(const Grid& g, const double* pos, int cap, const int* counters, int* key, int* hist, int* ord,
                    int* rank, cudaStream_t s) {
    static_assert(BS_SORT_MIN >= 342 && BS_SORT_MAX_BINS <= 256, "the bin counts must fit in cap ints");
    const BsBins bb = bs_bins(g.nx, g.ny, g.nz);
    const int nblk = (cap + SORT_BLOCK - 1) / SORT_BLOCK > 0 ? (cap + SORT_BLOCK - 1) / SORT_BLOCK : 1;
    launch_pdl(k_sort_count, nblk, SORT_BLOCK, 0, s, g, bb, pos, cap, counters, key, hist, nblk);
    launch_pdl(k_sort_scan, 1, 1024, 0, s, bb.K * nblk, hist);
    launch_pdl(k_sort_place, nblk, SORT_BLOCK, 0, s, bb.K, counters, (const int*)key, (const int*)hist, nblk, ord,
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
