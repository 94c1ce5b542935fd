// Filament topology updates of the coupled step (Sec. II.A of
// arXiv 2108.04435): remeshing to the resolution [dxi_min, dxi_max] and
// reconnection by leg exchange when two vortices come within dxi_max
// (Sec. III.B), then deletion of loops with fewer than five points and a
// stable compaction of the point arrays.
//
// Rules (the paper fixes only the resolution and "exchange the legs"):
//  remesh    split every segment longer than dxi_max at its arc midpoint
//            s_i + b/2 - (l^2/16)(s''_i + s''_q) (new points appended in
//            ascending i); a point with a neighbouring segment shorter than
//            dxi_min whose removal keeps the merged segment within dxi_max,
//            and whose segments are not split, is removed unless a candidate
//            neighbour outranks it (fmix32 priority of the index).
//  reconnect nearest j of each i within dxi_max outside its two-link
//            neighbourhood (ties to the smaller j); for mutual pairs the first
//            of the segment pairs (i,j), (i,p(j)), (p(i),j), (p(i),p(j)) with
//            the largest positive length decrease is exchanged; exchanges are
//            applied in ascending (d^2, i), skipping any that touches a point
//            already used; a pair whose segment is missing (a line's last
//            point) is not tried.
//  walls     open lines end on walls: an end keeps the mirror image of its
//            neighbour across its wall as the missing neighbour and is never
//            removed; after the exchanges a point with both neighbours that
//            touches a wall's clamp bound cuts its line there (ascending
//            index, skipping points already used): it is deleted and its
//            neighbours become ends moved onto that bound.  Loops and lines
//            of fewer than five points are deleted.
// All decisions are FP64 predicates evaluated in the same order as a plain
// IEEE implementation (this file is compiled with -fmad=false), so they are
// bit-identical to it on identical inputs.
#include <cuda_runtime.h>
#include <math.h>

#include "vlb_internal.cuh"

namespace vlb {

namespace {

__device__ __forceinline__ double min_image(const Grid& g, int axis, double d) {
    if (!g.wall[axis]) {
        const double L = (double)(axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz));
        if (d > 0.5 * L) d -= L;
        else if (d < -0.5 * L) d += L;
    }
    return d;
}

__device__ __forceinline__ double dist(const Grid& g, const double* pos, int cap, int from, int to) {
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = min_image(g, k, pos[(long long)k * cap + to] - pos[(long long)k * cap + from]);
    return sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
}

__device__ __forceinline__ double wall_bound(const Grid& g, double dmin, int code) {
    const int a = code >> 1;
    const double L = (double)(a == 0 ? g.nx : (a == 1 ? g.ny : g.nz));
    return (code & 1) ? L - 0.5 - 0.5 * dmin : -0.5 + 0.5 * dmin;
}

// First wall clamp bound touched by point i (order x-, x+, y-, y+, z-, z+) as
// 2*axis + side, or -1.
__device__ __forceinline__ int touching_wall(const Grid& g, double dmin, const double* pos, int cap, int i) {
    for (int a = 0; a < 3; ++a) {
        if (!g.wall[a]) continue;
        const double x = pos[(long long)a * cap + i];
        if (x <= wall_bound(g, dmin, 2 * a)) return 2 * a;
        if (x >= wall_bound(g, dmin, 2 * a + 1)) return 2 * a + 1;
    }
    return -1;
}

// MurmurHash3 32-bit finaliser (fmix32), used as the merge priority.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ bool outranks(int a, int b) {
    const uint32_t ha = fmix32((uint32_t)a), hb = fmix32((uint32_t)b);
    return ha > hb || (ha == hb && a < b);
}

// Block-wide exclusive scan of one int per thread (blockDim.x == 1024).
__device__ int block_exclusive_scan(int v, int* total) {
    __shared__ int warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = warp_sums[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    const int base = wid > 0 ? warp_sums[wid - 1] : 0;
    const int tot = warp_sums[31];
    __syncthreads();
    *total = tot;
    return base + x - v;
}

// FP64 geometry for the remeshing decisions: segment length l+ = |s_q - s_i|
// and the three-point curvature s'' = 2 (l- b - l+ a) / (l+ l- (l+ + l-)) on
// the non-uniform arc-length grid (a = s_i - s_p, b = s_q - s_i); an open
// end on a wall uses the mirror image of its neighbour across the wall, and a
// line's last point has seglen 0.
__device__ __forceinline__ bool geometry_exact_point(const VfmParams& P, const double* __restrict__ s,
                                                     const int* __restrict__ next, const int* __restrict__ prev,
                                                     int cap, int i, double* __restrict__ spp,
                                                     double* __restrict__ seglen, uint8_t* __restrict__ flags) {
    const int p = prev[i], q = next[i];
    const int pl = p >= 0 ? p : i, ql = q >= 0 ? q : i;  // an end loads itself in place of the missing one
    double si[3], sp[3], sq[3], a[3], b[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        si[k] = s[(long long)k * cap + i];
        sp[k] = s[(long long)k * cap + pl];
        sq[k] = s[(long long)k * cap + ql];
    }
    int code = -1;
    if (p < 0 || q < 0) {
        code = touching_wall(P.g, P.dmin, s, cap, i);
        const int ax = code >> 1;
        const double L = (double)(ax == 0 ? P.g.nx : (ax == 1 ? P.g.ny : P.g.nz));
        const double w = (code & 1) ? L - 0.5 : -0.5;
#pragma unroll
        for (int k = 0; k < 3; ++k) {  // the mirror image of the present neighbour across the wall
            if (p < 0) sp[k] = k == ax ? 2.0 * w - sq[k] : sq[k];
            else sq[k] = k == ax ? 2.0 * w - sp[k] : sp[k];
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a[k] = min_image(P.g, k, si[k] - sp[k]);
        b[k] = min_image(P.g, k, sq[k] - si[k]);
    }
    if (code < 0 && (p < 0 || q < 0)) {  // an end on no wall is continued straight
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (p < 0) a[k] = b[k];
            else b[k] = a[k];
        }
    }
    const double lm = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    const double lp = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    const double den = lp * lm * (lp + lm);
    for (int k = 0; k < 3; ++k) spp[(long long)k * cap + i] = 2.0 * (lm * b[k] - lp * a[k]) / den;
    seglen[i] = q >= 0 ? lp : 0.0;
    // Remesh flags (bit 1 split, bit 2 removal candidate).  The predecessor's
    // segment length is lm: the same expression its own thread evaluates.
    const bool split = q >= 0 && lp > P.dmax;
    bool cand = false;
    if (p >= 0 && q >= 0) {  // open ends are never removed
        const bool split_p = lm > P.dmax;
        const double lmin = lm < lp ? lm : lp;
        double d[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) d[k] = min_image(P.g, k, sq[k] - sp[k]);
        const double lpq = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        cand = (lmin < P.dmin) && (lpq <= P.dmax) && !split_p && !split;
    }
    flags[i] = (uint8_t)((split ? 1 : 0) | (cand ? 2 : 0));
    return split || cand;
}

__global__ void __launch_bounds__(64) k_geometry_exact(VfmParams P, const double* __restrict__ s,
                                                       const int* __restrict__ next, const int* __restrict__ prev,
                                                       int* __restrict__ counters, int cap,
                                                       double* __restrict__ spp, double* __restrict__ seglen,
                                                       uint8_t* __restrict__ flags) {
    pdl_wait_trigger();
    const int N = counters[CNT_N];
    bool any = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        any |= geometry_exact_point(P, s, next, prev, cap, i, spp, seglen, flags);
    if (__ballot_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) atomicOr(&counters[CNT_RFLAGS], 1);
}

// ------------------------------------------------------------------ remesh

// Points of loops and open lines with fewer than five points die; one block,
// strided over [0, T).  A loop point finds its own loop (succ^k(i) == i,
// k <= 4); a line is measured and deleted by the thread of its first point
// (start(k) says which points have no predecessor).  Returns this thread's
// count.
template <typename StartFn>
__device__ int block_small_components(const int* __restrict__ succ, uint8_t* __restrict__ alive, int T,
                                      StartFn start, int* __restrict__ counters) {
    int dead = 0;
    for (int k = threadIdx.x; k < T; k += blockDim.x) {
        if (!alive[k]) continue;
        if (start(k)) {
            int j = k, size = 1;
            while (size < 5) {
                const int n = succ[j];
                if (n < 0) break;
                if (n >= T) {
                    atomicOr(&counters[CNT_STATUS], ST_TOPOLOGY);
                    size = 5;
                    break;
                }
                j = n;
                ++size;
            }
            if (size < 5)
                for (j = k; j >= 0; j = succ[j]) {
                    alive[j] = 0;
                    ++dead;
                }
            continue;
        }
        int j = k;
        for (int s = 1; s <= 4; ++s) {
            j = succ[j];
            if (j < 0) break;  // a line, handled from its first point
            if (j >= T) {
                atomicOr(&counters[CNT_STATUS], ST_TOPOLOGY);
                break;
            }
            if (j == k) {
                alive[k] = 0;
                ++dead;
                break;
            }
        }
    }
    return dead;
}

// One block: stable compaction of the alive points of [0, T) into the other
// point buffer, successor indices renumbered, predecessors rebuilt.  The
// points go in chunks of blockDim.x consecutive indices, one per thread: a
// ballot per warp and a scan over the warps rank the alive points of a chunk,
// so every load and store of a chunk is coalesced (per-thread ranges of
// consecutive points made each warp access touch 32 lines).
__device__ void block_compact(const double* __restrict__ pin, const int* __restrict__ succ,
                              const uint8_t* __restrict__ alive, int T, int* __restrict__ newidx,
                              double* __restrict__ pout, int* __restrict__ nout, int* __restrict__ pvout,
                              int* __restrict__ counters, int cap) {
    __shared__ int s_off[33];  // per-warp exclusive offsets of a chunk; [32] = the chunk's count
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)blockDim.x >> 5;
    int M = 0;
    for (int c0 = 0; c0 < T; c0 += blockDim.x) {
        const int k = c0 + (int)threadIdx.x;
        const bool a = k < T && alive[k] != 0;
        const unsigned m = __ballot_sync(0xffffffffu, a);
        if (lane == 0) s_off[wid] = __popc(m);
        __syncthreads();
        if (wid == 0) {
            const int v = lane < nw ? s_off[lane] : 0;
            int x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane < nw) s_off[lane] = x - v;
            if (lane == 31) s_off[32] = x;
        }
        __syncthreads();
        if (k < T) {
            const int n = a ? M + s_off[wid] + __popc(m & ((1u << lane) - 1u)) : -1;
            newidx[k] = n;
            if (a) pvout[n] = -1;  // first points of lines keep -1
        }
        M += s_off[32];
        __syncthreads();  // s_off is reused by the next chunk
    }
    for (int k = threadIdx.x; k < T; k += blockDim.x) {
        if (!alive[k]) continue;
        const int n = newidx[k];
        for (int c = 0; c < 3; ++c) pout[(long long)c * cap + n] = pin[(long long)c * cap + k];
        const int sk = succ[k];
        if (sk < 0) {  // last point of an open line
            nout[n] = -1;
            continue;
        }
        const int sn = sk < T ? newidx[sk] : -1;
        if (sn < 0) {
            atomicOr(&counters[CNT_STATUS], ST_TOPOLOGY);
            continue;
        }
        nout[n] = sn;
        pvout[sn] = n;
    }
    __syncthreads();
    if (threadIdx.x == 0) counters[CNT_N] = M;
}

// The points and links of [0, N) copied unchanged into the other point
// buffer, when the topology finish before found nothing to change
// (counters[CNT_PASS], which that finish sets either way): the finish itself
// is one block, and one block moving the whole point set is bound by memory
// latency (~80 us for 86k points), a grid by bandwidth.
__global__ void k_points_pass(const int* __restrict__ counters, const double* __restrict__ pin,
                              const int* __restrict__ succ, const int* __restrict__ pred, double* __restrict__ pout,
                              int* __restrict__ nout, int* __restrict__ pvout, int* __restrict__ newidx, int cap) {
    pdl_wait_trigger();
    if (!counters[CNT_PASS]) return;
    const int N = counters[CNT_N];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        pout[k] = pin[k];
        pout[(long long)cap + k] = pin[(long long)cap + k];
        pout[2LL * cap + k] = pin[2LL * cap + k];
        nout[k] = succ[k];
        pvout[k] = pred[k];
        newidx[k] = k;
    }
}

__device__ int block_sum(int v) {
    __shared__ int s_red[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[wid] = v;
    __syncthreads();
    int t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
    __syncthreads();
    return t;  // valid in thread 0
}

// One block finishes the remesh: ranks of the split segments (ascending i),
// removals, the new points' positions and successors, small-loop deletion and
// the compaction into the other point buffer.
__global__ void __launch_bounds__(1024) k_remesh_finish(VfmParams P, double* __restrict__ pos,
                                                         const int* __restrict__ next, const int* __restrict__ prev,
                                                         const double* __restrict__ spp,
                                                         const double* __restrict__ seglen,
                                                         const uint8_t* __restrict__ flags, int* __restrict__ nnext,
                                                         uint8_t* __restrict__ alive, int* __restrict__ newidx,
                                                         double* __restrict__ pout, int* __restrict__ nout,
                                                         int* __restrict__ pvout, int* __restrict__ counters,
                                                         double* __restrict__ dstats, int cap) {
    pdl_wait_trigger();
    const int N = counters[CNT_N];
    __shared__ int s_any;
    if (threadIdx.x == 0) {
        s_any = counters[CNT_RFLAGS] | counters[CNT_DIRTY];
        counters[CNT_RFLAGS] = 0;
    }
    __syncthreads();
    if (!s_any) {
        // no split, no removal candidate and nothing newly seeded: the points
        // and links pass through unchanged (what the full pass concludes
        // too), copied by k_points_pass
        if (threadIdx.x == 0) counters[CNT_PASS] = 1;
        return;
    }
    const int per = (N + (int)blockDim.x - 1) / (int)blockDim.x;
    const int b0 = min(N, (int)threadIdx.x * per);
    const int b1 = min(N, b0 + per);
    int mine = 0;
    for (int i = b0; i < b1; ++i) mine += flags[i] & 1;
    int S = 0;
    int running = block_exclusive_scan(mine, &S);
    if ((long long)N + S > (long long)cap) {
        if (threadIdx.x == 0) atomicOr(&counters[CNT_STATUS], ST_CAPACITY);
        S = 0;
    }
    int removed = 0;
    for (int i = b0; i < b1; ++i) {
        const uint8_t fi = flags[i];
        const int p = prev[i], q = next[i];
        const bool rem = (fi & 2) && !((flags[p] & 2) && outranks(p, i)) && !((flags[q] & 2) && outranks(q, i));
        alive[i] = rem ? 0 : 1;
        if (rem) {
            ++removed;
            continue;
        }
        if (q < 0) {
            nnext[i] = -1;
        } else if ((fi & 1) && S > 0) {
            const int m = N + running;
            const double l = seglen[i];
            double ms[3];
            for (int k = 0; k < 3; ++k) {
                const long long oi = (long long)k * cap + i, oq = (long long)k * cap + q;
                const double b = min_image(P.g, k, pos[oq] - pos[oi]);
                ms[k] = pos[oi] + 0.5 * b - (l * l / 16.0) * (spp[oi] + spp[oq]);
            }
            for (int a = 0; a < 3; ++a) {
                const double L = (double)(a == 0 ? P.g.nx : (a == 1 ? P.g.ny : P.g.nz));
                if (!P.g.wall[a]) {
                    if (ms[a] < 0.0) ms[a] += L;
                    else if (ms[a] >= L) ms[a] -= L;
                } else {
                    const double lo = -0.5 + 0.5 * P.dmin, hi = L - 0.5 - 0.5 * P.dmin;
                    if (ms[a] < lo) ms[a] = lo;
                    if (ms[a] > hi) ms[a] = hi;
                }
                pos[(long long)a * cap + m] = ms[a];
            }
            nnext[i] = m;
            nnext[m] = q;
            alive[m] = 1;
        } else {
            const uint8_t fq = flags[q];
            const int qp = i, qn = next[q];
            const bool rem_q =
                (fq & 2) && !((flags[qp] & 2) && outranks(qp, q)) && !((flags[qn] & 2) && outranks(qn, q));
            nnext[i] = rem_q ? qn : q;
        }
        if (fi & 1) ++running;
    }
    const int T = N + S;
    __syncthreads();
    // Splits only add points, so without removals no loop or line shrinks
    // below five points here (every one had five or more after the last
    // reconnection pass), unless the points were just seeded.
    __shared__ int s_check;
    const int removed_all = block_sum(removed);
    if (threadIdx.x == 0) {
        s_check = removed_all > 0 || counters[CNT_DIRTY] != 0;
        counters[CNT_DIRTY] = 0;
    }
    __syncthreads();
    const int dead = s_check ? block_small_components(
                                   nnext, alive, T, [&](int k) { return k < N && prev[k] < 0; }, counters)
                             : 0;
    const int dead_all = block_sum(dead);
    __shared__ int s_same;  // no split, removal or deletion: points and links pass through unchanged
    if (threadIdx.x == 0) {
        dstats[DS_SPLITS] += (double)S;
        dstats[DS_MERGES] += (double)removed_all;
        dstats[DS_SMALL] += (double)dead_all;
        s_same = S == 0 && removed_all == 0 && dead_all == 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) counters[CNT_PASS] = s_same ? 1 : 0;
    if (s_same) return;  // (nnext equals next then) copied by k_points_pass
    block_compact(pos, nnext, alive, T, newidx, pout, nout, pvout, counters, cap);
}

// -------------------------------------------------------------- reconnect

__device__ __forceinline__ uint32_t cell_hash(int cx, int cy, int cz) {
    return ((uint32_t)cx * 73856093u) ^ ((uint32_t)cy * 19349663u) ^ ((uint32_t)cz * 83492791u);
}

// Unit-cell hash of the points: bucket heads (kept at -1 between passes) and a
// link per point, filled with atomicExch; bucket order does not matter.  The
// link is also stored beside the point's FP32 position in hpos, the record
// the nearest-point search walks.
__global__ void k_hash_insert(const double* __restrict__ pos, int* __restrict__ counters, int cap,
                              uint32_t hmask, int* __restrict__ hkey, int* __restrict__ hhead,
                              int* __restrict__ hlink, float4* __restrict__ hpos) {
    pdl_wait_trigger();
    const int N = counters[CNT_N];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        counters[CNT_NPAIRS] = 0;
        counters[CNT_NCONTACT] = 0;
    }
    for (int i = t; i < N; i += gridDim.x * blockDim.x) {
        const double x = pos[i], y = pos[(long long)cap + i], z = pos[2LL * cap + i];
        const int h = (int)(cell_hash((int)floor(x), (int)floor(y), (int)floor(z)) & hmask);
        hkey[i] = h;
        const int link = atomicExch(&hhead[h], i);
        hlink[i] = link;
        hpos[i] = make_float4(__double2float_rn(x), __double2float_rn(y), __double2float_rn(z), __int_as_float(link));
    }
}

__device__ __forceinline__ float min_image_f(const Grid& g, int axis, float d) {
    if (!g.wall[axis]) {
        const float L = (float)(axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz));
        if (d > 0.5f * L) d -= L;
        else if (d < -0.5f * L) d += L;
    }
    return d;
}

// Nearest point within dxi_max outside the two-link neighbourhood.  Every
// point closer than dxi_max < 1 lies in one of the 27 unit cells around; one
// warp per point, lane l < 27 walks the bucket of cell l, then the warp takes
// the minimum of (d^2, j).  The walk reads the FP32 records of hpos and skips
// a point whose FP32 distance squared exceeds r2f, a bound above which the
// FP64 distance is certainly not below dxi_max (nearest_filter_r2); the
// others are decided in FP64 exactly as without the filter.
__global__ void __launch_bounds__(128) k_nearest(VfmParams P, double dmax2, float r2f, const double* __restrict__ pos,
                                                 const int* __restrict__ next, const int* __restrict__ prev,
                                                 const int* __restrict__ counters, int cap, uint32_t hmask,
                                                 const int* __restrict__ hhead, const float4* __restrict__ hpos,
                                                 int* __restrict__ nn, double* __restrict__ nd2) {
    pdl_wait_trigger();
    const int N = counters[CNT_N];
    const int lane = threadIdx.x & 31, wpb = (int)(blockDim.x >> 5);
    // one point per warp at a time: i is uniform over the warp
    for (int i = (int)blockIdx.x * wpb + (int)(threadIdx.x >> 5); i < N; i += (int)gridDim.x * wpb) {
        const int p = prev[i], q = next[i], pp = p >= 0 ? prev[p] : -1, qq = q >= 0 ? next[q] : -1;
        const float4 fi = hpos[i];
        int best = -1;
        double bd = 0.0;
        if (lane < 27) {
            double xi[3];
            int c[3];
            for (int k = 0; k < 3; ++k) {
                xi[k] = pos[(long long)k * cap + i];
                c[k] = (int)floor(xi[k]);
            }
            const int n[3] = {P.g.nx, P.g.ny, P.g.nz};
            int cc[3] = {c[0] + lane % 3 - 1, c[1] + (lane / 3) % 3 - 1, c[2] + lane / 9 - 1};
            for (int a = 0; a < 3; ++a)
                if (!P.g.wall[a]) cc[a] = ((cc[a] % n[a]) + n[a]) % n[a];
            const int h = (int)(cell_hash(cc[0], cc[1], cc[2]) & hmask);
            int j = hhead[h];
            for (int guard = 0; j >= 0 && guard < N; ++guard) {
                const float4 fj = hpos[j];
                const int jn = __float_as_int(fj.w);
                const float e0 = min_image_f(P.g, 0, fj.x - fi.x), e1 = min_image_f(P.g, 1, fj.y - fi.y),
                            e2 = min_image_f(P.g, 2, fj.z - fi.z);
                const bool skip = j == i || j == p || j == q || j == pp || j == qq || e0 * e0 + e1 * e1 + e2 * e2 > r2f;
                if (!skip) {
                    double d[3];
                    for (int k = 0; k < 3; ++k) d[k] = min_image(P.g, k, pos[(long long)k * cap + j] - xi[k]);
                    const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (d2 < dmax2 && (best < 0 || d2 < bd || (d2 == bd && j < best))) {
                        best = j;
                        bd = d2;
                    }
                }
                j = jn;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int ob = __shfl_xor_sync(0xffffffffu, best, o);
            const double od = __shfl_xor_sync(0xffffffffu, bd, o);
            if (ob >= 0 && (best < 0 || od < bd || (od == bd && ob < best))) {
                best = ob;
                bd = od;
            }
        }
        if (lane == 0) {
            nn[i] = best;
            nd2[i] = bd;
        }
    }
}

// Candidate exchanges of the mutual nearest pairs, and the wall-contact
// candidates (points with both neighbours on a wall's clamp bound; exchanges
// change neither property), each appended to its list.  Four threads per
// point: thread k of the quad evaluates the k-th exchange (i,j), (i,p(j)),
// (p(i),j), (p(i),p(j)) (its four FP64 distances); the quad keeps the largest
// positive gain, the lowest k among equal gains, which is what evaluating the
// four in order and keeping a strictly larger gain selects.
__global__ void k_pairs(VfmParams P, const double* __restrict__ pos, const int* __restrict__ next,
                        const int* __restrict__ prev, const int* __restrict__ nn, const double* __restrict__ nd2,
                        int* __restrict__ counters, int cap, int* __restrict__ cand_i, int* __restrict__ cand_a,
                        int* __restrict__ cand_b, double* __restrict__ cand_d2, int* __restrict__ clist,
                        const int* __restrict__ hkey, int* __restrict__ hhead) {
    pdl_wait_trigger();
    const int N = counters[CNT_N];
    const int k = threadIdx.x & 3;
    // the nearest-point search is done with the hash: empty its buckets for
    // the next pass (a grid clears them at memory speed; one block would not)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) hhead[hkey[i]] = -1;
    const unsigned quad = 0xfu << (threadIdx.x & 28);
    const int nq = (int)((gridDim.x * blockDim.x) >> 2);
    // i is uniform over a quad, so each quad runs the loop and its shuffles together
    for (int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 2); i < N; i += nq) {
        const int pi = prev[i];
        if (k == 0 && (P.g.wall[0] | P.g.wall[1] | P.g.wall[2])) {
            if (pi >= 0 && next[i] >= 0 && touching_wall(P.g, P.dmin, pos, cap, i) >= 0)
                clist[atomicAdd(&counters[CNT_NCONTACT], 1)] = i;
        }
        const int j = nn[i];
        if (j <= i || nn[j] != i) continue;
        const int pj = prev[j];
        const int a = k < 2 ? i : pi, b = (k & 1) ? pj : j;
        bool ok = false;
        double gain = 0.0;
        if (a >= 0 && b >= 0) {
            const int qa = next[a], qb = next[b];
            if (qa >= 0 && qb >= 0) {
                gain = (dist(P.g, pos, cap, a, qa) + dist(P.g, pos, cap, b, qb)) -
                       (dist(P.g, pos, cap, a, qb) + dist(P.g, pos, cap, b, qa));
                ok = gain > 0.0;
            }
        }
        int kb = ok ? k : 4;  // 4: no exchange
#pragma unroll
        for (int o = 1; o < 4; o <<= 1) {
            const double og = __shfl_xor_sync(quad, gain, o);
            const int ok_ = __shfl_xor_sync(quad, kb, o);
            if (ok_ < 4 && (kb == 4 || og > gain || (og == gain && ok_ < kb))) {
                gain = og;
                kb = ok_;
            }
        }
        if (k != 0 || kb == 4) continue;
        const int slot = atomicAdd(&counters[CNT_NPAIRS], 1);
        cand_i[slot] = i;
        cand_a[slot] = kb < 2 ? i : pi;
        cand_b[slot] = (kb & 1) ? pj : j;
        cand_d2[slot] = nd2[i];
    }
}

// One block finishes the reconnection: candidates in ascending (d^2, i)
// order (keys are unique), the greedy pass in that order (an exchange that
// touches a point already used is skipped), the wall-contact cuts,
// small-component deletion and the compaction into the other point buffer;
// when nothing changes, k_points_pass copies the points instead (the hash
// buckets were emptied by k_pairs).
__global__ void __launch_bounds__(1024) k_reconnect_finish(
    VfmParams P, const int* __restrict__ clist, double* __restrict__ pos, int* __restrict__ next,
    int* __restrict__ prev, const int* __restrict__ cand_i,
    const int* __restrict__ cand_a, const int* __restrict__ cand_b, const double* __restrict__ cand_d2,
    int* __restrict__ order, int* __restrict__ stamp,
    uint8_t* __restrict__ alive, int* __restrict__ newidx, double* __restrict__ pout, int* __restrict__ nout,
    int* __restrict__ pvout, int* __restrict__ counters, double* __restrict__ dstats, int cap) {
    pdl_wait_trigger();
    const int N = counters[CNT_N];
    const int K = counters[CNT_NPAIRS];
    __shared__ int s_quiet;
    if (threadIdx.x == 0) s_quiet = K == 0 && counters[CNT_NCONTACT] == 0 && counters[CNT_DIRTY] == 0;
    __syncthreads();
    if (s_quiet) {
        // no candidate exchange, no wall contact and nothing newly seeded:
        // the points and links pass through (copied by k_points_pass)
        if (threadIdx.x == 0) {
            counters[CNT_STAMP] += 1;
            counters[CNT_PASS] = 1;
        }
        return;
    }
    for (int c = threadIdx.x; c < K; c += blockDim.x) {
        const double d = cand_d2[c];
        const int ic = cand_i[c];
        int r = 0;
        for (int o = 0; o < K; ++o) {
            const double e = cand_d2[o];
            r += (e < d || (e == d && cand_i[o] < ic)) ? 1 : 0;
        }
        order[r] = c;
    }
    for (int k = threadIdx.x; k < N; k += blockDim.x) alive[k] = 1;
    __shared__ int s_changed;  // an exchange or a cut happened: small components may have formed
    __syncthreads();
    if (threadIdx.x == 0) {
        const int st = counters[CNT_STAMP] + 1;
        counters[CNT_STAMP] = st;
        int applied = 0;
        for (int r = 0; r < K; ++r) {
            const int c = order[r];
            const int a = cand_a[c], b = cand_b[c];
            const int qa = next[a], qb = next[b];
            if (stamp[a] == st || stamp[qa] == st || stamp[b] == st || stamp[qb] == st) continue;
            stamp[a] = st;
            stamp[qa] = st;
            stamp[b] = st;
            stamp[qb] = st;
            next[a] = qb;
            prev[qb] = a;
            next[b] = qa;
            prev[qa] = b;
            ++applied;
        }
        dstats[DS_RECON] += (double)applied;
        s_changed = applied > 0 || counters[CNT_DIRTY] != 0;  // (seeded points not yet remeshed: check them)
        counters[CNT_DIRTY] = 0;
    }
    __syncthreads();
    // Wall contact: the candidates listed by k_pairs, put in ascending index
    // order (indices are unique; newidx holds the order until the compaction),
    // then cut in that order by one thread.
    int* corder = newidx;
    const int ncand = counters[CNT_NCONTACT];
    for (int c = threadIdx.x; c < ncand; c += blockDim.x) {
        const int ic = clist[c];
        int r = 0;
        for (int o = 0; o < ncand; ++o) r += clist[o] < ic ? 1 : 0;
        corder[r] = ic;
    }
    __syncthreads();
    if (threadIdx.x == 0 && ncand > 0) {
        const int st = counters[CNT_STAMP];
        int cuts = 0;
        for (int r = 0; r < ncand; ++r) {
            const int i = corder[r], p = prev[i], q = next[i];
            if (stamp[i] == st || stamp[p] == st || stamp[q] == st) continue;
            const int code = touching_wall(P.g, P.dmin, pos, cap, i);
            stamp[i] = st;
            stamp[p] = st;
            stamp[q] = st;
            alive[i] = 0;
            next[p] = -1;
            prev[q] = -1;
            const double bnd = wall_bound(P.g, P.dmin, code);
            pos[(long long)(code >> 1) * cap + p] = bnd;
            pos[(long long)(code >> 1) * cap + q] = bnd;
            ++cuts;
        }
        dstats[DS_WALLCUT] += (double)cuts;
        if (cuts > 0) s_changed = 1;
    }
    __syncthreads();
    const int dead =
        s_changed ? block_small_components(next, alive, N, [&](int k) { return prev[k] < 0; }, counters) : 0;
    const int dead_all = block_sum(dead);
    if (threadIdx.x == 0) dstats[DS_SMALL] += (double)dead_all;
    __syncthreads();
    // no exchange and no cut: the points and links pass through unchanged
    // (copied by k_points_pass)
    if (threadIdx.x == 0) counters[CNT_PASS] = s_changed ? 0 : 1;
    if (!s_changed) return;
    block_compact(pos, next, alive, N, newidx, pout, nout, pvout, counters, cap);
}

}  // namespace

void launch_remesh_geometry(const VfmParams& P, Dev& d, int cur, int cap, int span, cudaStream_t s) {
    if (cap <= 0) return;
    launch_pdl(k_geometry_exact, (span + 63) / 64, 64, 0, s, P, d.pos[cur], d.next[cur], d.prev[cur], d.counters, cap,
               d.spp, d.seglen, d.flags);
}

// After a finish: the unchanged points into the other buffer, if the finish
// passed them through (a grid-stride kernel of four blocks per SM).
static void launch_points_pass(Dev& d, int cur, int cap, cudaStream_t s) {
    launch_pdl(k_points_pass, 4 * sm_count(), 256, 0, s, (const int*)d.counters, (const double*)d.pos[cur],
               (const int*)d.next[cur], (const int*)d.prev[cur], d.pos[cur ^ 1], d.next[cur ^ 1], d.prev[cur ^ 1],
               d.newidx, cap);
}

void launch_remesh_finish(const VfmParams& P, Dev& d, int cur, int cap, cudaStream_t s) {
    if (cap <= 0) return;
    launch_pdl(k_remesh_finish, 1, 1024, 0, s, P, d.pos[cur], d.next[cur], d.prev[cur], d.spp, d.seglen, d.flags, d.nnext,
                                       d.alive, d.newidx, d.pos[cur ^ 1], d.next[cur ^ 1], d.prev[cur ^ 1],
                                       d.counters, d.dstats, cap);
    launch_points_pass(d, cur, cap, s);
}

void launch_remesh(const VfmParams& P, Dev& d, int cur, int cap, int span, cudaStream_t s) {
    launch_remesh_geometry(P, d, cur, cap, span, s);
    launch_remesh_finish(P, d, cur, cap, s);
}

void init_hash(Dev& d, int hsize, cudaStream_t s) { cudaMemsetAsync(d.hhead, 0xff, sizeof(int) * (size_t)hsize, s); }

// The FP32 bound of the nearest-point search.  Positions lie within
// [-0.5, L] on every axis (L the largest extent), so the FP32 roundings of
// the two coordinates, of their difference and of the periodic shift err by
// at most 5 L 2^-24 on an axis together: an FP32 distance vector is within
// 5 sqrt(3) L 2^-24 < 9 L 2^-24 of the FP64 one, wherever both take the same
// periodic image.  Where they
// take different images (a difference within that error of L/2), both
// distances are near L/2 > dxi_max + the margin, which holds when every
// periodic extent is 4 or more; otherwise the filter is off.  The bound
// (dxi_max + 16 L 2^-24)^2 (1 + 2^-20), rounded up to FP32, also covers the
// roundings of the squared sum.
float nearest_filter_r2(const VfmParams& P) {
    const int n[3] = {P.g.nx, P.g.ny, P.g.nz};
    double L = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (!P.g.wall[a] && n[a] < 4) return INFINITY;
        L = fmax(L, (double)n[a]);
    }
    const double r = P.dmax + 16.0 * L * ldexp(1.0, -24);
    const float r2 = (float)(r * r * (1.0 + ldexp(1.0, -20)));
    return nextafterf(r2, INFINITY);
}

void launch_reconnect(const VfmParams& P, Dev& d, int cur, int cap, int span, int hsize, cudaStream_t s) {
    if (cap <= 0) return;
    const uint32_t hmask = (uint32_t)hsize - 1u;
    const double dmax2 = P.dmax * P.dmax;
    launch_pdl(k_hash_insert, (span + 255) / 256, 256, 0, s, d.pos[cur], d.counters, cap, hmask, d.hkey, d.hhead, d.hlink,
               d.hpos);
    launch_pdl(k_nearest, (span + 3) / 4, 128, 0, s, P, dmax2, nearest_filter_r2(P), d.pos[cur], d.next[cur], d.prev[cur],
               d.counters, cap, hmask, d.hhead, d.hpos, d.nn, d.nd2);
    launch_pdl(k_pairs, (4 * span + 127) / 128, 128, 0, s, P, d.pos[cur], d.next[cur], d.prev[cur], d.nn, d.nd2,
               d.counters, cap, d.cand_i, d.cand_a, d.cand_b, d.cand_d2, d.hlink, d.hkey, d.hhead);
    launch_pdl(k_reconnect_finish, 1, 1024, 0, s, P, d.hlink, d.pos[cur], d.next[cur], d.prev[cur], d.cand_i, d.cand_a, d.cand_b,
                                          d.cand_d2, d.cand_order, d.stamp, d.alive, d.newidx,
                                          d.pos[cur ^ 1], d.next[cur ^ 1], d.prev[cur ^ 1], d.counters, d.dstats,
                                          cap);
    launch_points_pass(d, cur, cap, s);
}

}  // namespace vlb
