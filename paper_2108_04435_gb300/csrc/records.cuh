// Biot-Savart source records (layout in vlb_internal.cuh): written by the
// stage geometry (vfm.cu) and by the stand-alone entry (bs.cu).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "vlb_internal.cuh"

namespace vlb {

namespace {

// The 16 values of one Biot-Savart source record (layout in
// vlb_internal.cuh): rel = the segment's start relative to its group origin
// (FP64), d = the segment.
__device__ __forceinline__ void bs_record_values(const double rel[3], const float d[3], float val[16]) {
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
    val[13] = val[14] = val[15] = 0.f;
}

// Store record k (scalar stores: its pair partner may belong to any thread).
__device__ __forceinline__ void bs_store_record(float4* __restrict__ seg, long long k, const float val[16]) {
    float* r = reinterpret_cast<float*>(seg);
#pragma unroll
    for (int v = 0; v < 16; ++v) r[bs_value_index(k, v)] = val[v];
}

__device__ __forceinline__ void bs_write_record(float4* __restrict__ seg, long long k, const double rel[3],
                                                const float d[3]) {
    float val[16];
    bs_record_values(rel, d, val);
    bs_store_record(seg, k, val);
}

// Store records k and k ^ 1, held by this lane and its neighbour lane ^ 1
// (k even on even lanes; all 32 lanes call it together): the two lanes swap
// half their values and each writes four of the pair's eight float4 (lane
// parity s writes float4 s, s + 2, s + 4, s + 6).  `has`: the pair lies
// inside the record block (the same for both lanes).
__device__ __forceinline__ void bs_store_pair(float4* __restrict__ seg, long long k, const float val[16], bool has) {
    const int s = threadIdx.x & 1;
    // float4 m of the pair holds (v_2m of record 0, of record 1, v_2m+1 of
    // record 0, of record 1); lane s needs the partner's values 2m, 2m + 1 for
    // m = s, s + 2, s + 4, s + 6, and sends those its partner needs
    float other[8];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int mine = 2 * (2 * j) + e, theirs = 2 * (2 * j + 1) + e;  // indices lane 0 / lane 1 wants
            const float send = s ? val[mine] : val[theirs];
            other[2 * j + e] = __shfl_xor_sync(0xffffffffu, send, 1);
        }
    if (!has) return;
    float4* P = seg + (k >> 1) * 8;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int m = 2 * j + s;
        const float a0 = val[2 * m], a1 = val[2 * m + 1], b0 = other[2 * j], b1 = other[2 * j + 1];
        P[m] = s ? make_float4(b0, a0, b1, a1) : make_float4(a0, b0, a1, b1);
    }
}

// Origin of group g in point order: the cell of its first point, point
// g * BS_GROUP (every thread of the group computes it from that point's
// position; the group's first thread also stores it for the Biot-Savart
// kernel, which reads org[]).
__device__ __forceinline__ int4 bs_point_order_origin(const double* __restrict__ s, int cap, int g, bool store,
                                                      int4* __restrict__ org) {
    const int i0 = g * BS_GROUP;
    const int4 O = make_int4((int)floor(s[i0]), (int)floor(s[(long long)cap + i0]), (int)floor(s[2LL * cap + i0]), 0);
    if (store) org[g] = O;
    return O;
}

// Record position and group origin of point i < N in the order o (positions
// s[3][cap], for the point-order origin).
__device__ __forceinline__ long long bs_position(const BsOrder& o, const double* __restrict__ s, int cap, int i,
                                                 double O[3]) {
    int4 g;
    long long k;
    if (o.sorted) {
        k = o.rank[i];
        g = o.org[k / BS_GROUP];
    } else {
        k = i;
        g = bs_point_order_origin(s, cap, i / BS_GROUP, i % BS_GROUP == 0, o.org);
    }
    O[0] = (double)g.x;
    O[1] = (double)g.y;
    O[2] = (double)g.z;
    return k;
}

// Zero-length records at the padding positions [N, Np) of every record block:
// thread i covers position i.
__device__ __forceinline__ void bs_pad_records(int N, int nfaces, int i, float4* __restrict__ seg) {
    const long long Np = bs_block(N, nfaces);
    if (i < N || i >= Np) return;
    const double z[3] = {0.0, 0.0, 0.0};
    const float d[3] = {0.f, 0.f, 0.f};
    for (int f = 0; f <= nfaces; ++f) bs_write_record(seg, (long long)f * Np + i, z, d);
}

}  // namespace

}  // namespace vlb
