// Biot-Savart source slots and target records (layouts in vlb_internal.cuh):
// written group by group by the stage geometry (vfm.cu) and by the
// stand-alone entry (bs.cu).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "eom.cuh"
#include "vlb_internal.cuh"

namespace vlb {

namespace {

// The values of one slot: rel = its point relative to the group origin
// (FP64), d = its segment (zero for none).
__device__ __forceinline__ void bs_slot_values(const double rel[3], const float d[3], float val[BS_VALS]) {
    float h[3], l[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        h[a] = __double2float_rn(rel[a]);
        l[a] = __double2float_rn(rel[a] - (double)h[a]);
    }
    val[0] = h[0]; val[1] = h[1]; val[2] = h[2];
    val[3] = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    val[4] = d[0]; val[5] = d[1]; val[6] = d[2];
    val[7] = h[1] * d[2] - h[2] * d[1];
    val[8] = h[2] * d[0] - h[0] * d[2];
    val[9] = h[0] * d[1] - h[1] * d[0];
    val[10] = l[0]; val[11] = l[1]; val[12] = l[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) val[13 + a] = __double2float_rn(rel[a] + (double)d[a]);
    val[16] = h[0] * h[0] + h[1] * h[1] + h[2] * h[2];
    val[17] = val[18] = val[19] = 0.f;
}

// The target record of the point at sorted position k (slot sl, parts h + l
// of its position in the group origin O, predecessor's slot, excluded image
// slot of a pinned end, point index i).
__device__ __forceinline__ void bs_write_target(float4* __restrict__ tgt, int k, const double rel[3], const int4& O,
                                                int sl, int prev_sl, int excl, int i) {
    float h[3], l[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        h[a] = __double2float_rn(rel[a]);
        l[a] = __double2float_rn(rel[a] - (double)h[a]);
    }
    float4* r = tgt + 4LL * k;
    r[0] = make_float4(h[0], h[1], h[2], l[0]);
    r[1] = make_float4(l[1], l[2], (float)O.x, (float)O.y);
    r[2] = make_float4((float)O.z, __int_as_float(sl), __int_as_float(prev_sl), __int_as_float(excl));
    r[3] = make_float4(__int_as_float(i), 0.f, 0.f, 0.f);
}

// Slot of the predecessor's segment (-1 for none).
__device__ __forceinline__ int bs_prev_slot(const BsOrder& o, int p) {
    return p >= 0 ? o.slot[o.sorted ? o.rank[p] : p] : -1;
}

// Shared memory of the group writer: one group's records in their stored
// layout, and the two warps' box partials.
struct BsGroupSmem {
    float stage[BS_GROUP * BS_VALS];
    float red[2][6];
};

// Centre a group's origin on its box of points (called by the whole block,
// thread t holding slot t's position rel relative to O): the origin moves by
// the integer cell nearest the box centre and rel with it (exactly), so
// that |h| stays within about half the group's extent.  Returns the new
// origin.
__device__ __forceinline__ int4 bs_center_origin(double rel[3], const int4& O, BsGroupSmem& sm) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) lo[a] = hi[a] = (float)rel[a];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], off));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], off));
        }
    if (lane == 0)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            sm.red[w][a] = lo[a];
            sm.red[w][3 + a] = hi[a];
        }
    __syncthreads();
    int sh[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        sh[a] = (int)rintf(0.5f * (fminf(sm.red[0][a], sm.red[1][a]) + fmaxf(sm.red[0][3 + a], sm.red[1][3 + a])));
        rel[a] -= (double)sh[a];
    }
    __syncthreads();  // sm.red is used again by the group writer
    return make_int4(O.x + sh[0], O.y + sh[1], O.z + sh[2], 0);
}

// One group of slots, written by one block of BS_GROUP threads, thread t =
// slot t of group grp: rel = its point relative to the group origin (FP64),
// d = its segment (zero for gap and padding slots), jump = the chain jumps
// by a periodic box between this slot and the next.  Writes the records of
// every record block (the segments, then one block per solid face:
// M(s) -> M(s) + M(d) with M mirroring the face axis, so each mirrored
// value is the direct one negated on that axis, exactly), with the group's
// box of h in the spare values 13-15 of slots 0 and 1 (low, high corner;
// unbounded when the chain jumps somewhere, which sends the group to the
// full-precision path), through shared memory in whole 16-byte stores.
__device__ __forceinline__ void bs_write_group(int nfaces, const int* face_code, long long Np, int grp,
                                               const double rel[3], const float d[3], bool jump, float4* seg,
                                               BsGroupSmem& sm) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    float val[BS_VALS];
    bs_slot_values(rel, d, val);
    float lo[3] = {val[0], val[1], val[2]}, hi[3] = {val[0], val[1], val[2]};
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], off));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], off));
        }
    if (lane == 0)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            sm.red[w][a] = lo[a];
            sm.red[w][3 + a] = hi[a];
        }
    const bool anyjump = __syncthreads_or(jump);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = anyjump ? -3.0e38f : fminf(sm.red[0][a], sm.red[1][a]);
        hi[a] = anyjump ? 3.0e38f : fmaxf(sm.red[0][3 + a], sm.red[1][3 + a]);
    }
    for (int f = 0; f <= nfaces; ++f) {
        float v[BS_VALS];
#pragma unroll
        for (int q = 0; q < BS_VALS; ++q) v[q] = val[q];
        float blo[3] = {lo[0], lo[1], lo[2]}, bhi[3] = {hi[0], hi[1], hi[2]};
        if (f > 0) {
            const int ax = face_code[f - 1] >> 1;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a != ax) continue;
                v[a] = -v[a];
                v[4 + a] = -v[4 + a];
                v[10 + a] = -v[10 + a];
                v[13 + a] = -v[13 + a];
                const float l0 = blo[a];
                blo[a] = -bhi[a];
                bhi[a] = -l0;
            }
            v[7] = v[1] * v[6] - v[2] * v[5];
            v[8] = v[2] * v[4] - v[0] * v[6];
            v[9] = v[0] * v[5] - v[1] * v[4];
        }
        if (t == 0) {
            v[13] = blo[0]; v[14] = blo[1]; v[15] = blo[2];
        } else if (t == 1) {
            v[13] = bhi[0]; v[14] = bhi[1]; v[15] = bhi[2];
        }
        // value q of slot t at (t % 32) * 2 BS_VALS + 2 q + (t / 32) of the group
#pragma unroll
        for (int q = 0; q < BS_VALS; ++q) sm.stage[lane * 2 * BS_VALS + 2 * q + w] = v[q];
        __syncthreads();
        float4* dst = seg + ((long long)f * Np + (long long)grp * BS_GROUP) * BS_REC;
        const float4* src = reinterpret_cast<const float4*>(sm.stage);
#pragma unroll
        for (int e = 0; e < BS_REC; ++e) dst[e * BS_GROUP + t] = src[e * BS_GROUP + t];
        __syncthreads();  // the stage is rewritten for the next block
    }
}

}  // namespace

}  // namespace vlb
