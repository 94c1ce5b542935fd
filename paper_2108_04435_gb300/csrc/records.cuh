// Biot-Savart source slots (layout in vlb_internal.cuh): written by the
// stage geometry (vfm.cu) and by the stand-alone entry (bs.cu).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "eom.cuh"
#include "vlb_internal.cuh"

namespace vlb {

namespace {

// The 16 values of one slot: rel = its point relative to the group origin
// (FP64), d = its segment (zero for none).
__device__ __forceinline__ void bs_slot_values(const double rel[3], const float d[3], float val[16]) {
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
}

// Store slot k (scalar stores: the other slot of its pair belongs to another
// thread).
__device__ __forceinline__ void bs_store_slot(float4* __restrict__ seg, long long k, const float val[16]) {
    float* r = reinterpret_cast<float*>(seg);
#pragma unroll
    for (int v = 0; v < 16; ++v) r[bs_value_index(k, v)] = val[v];
}

// Where the slots of one point go: its own slot k in the origin O of its
// group, and with `gap` the gap slot k + 1 (holding the successor) in the
// origin Og of that slot's group.
struct BsPointSlots {
    long long k;
    bool gap;
    double O[3], Og[3];
};

// Slots of the point at sorted position kk (point i, successor q or -1).
__device__ __forceinline__ BsPointSlots bs_point_slots(const BsOrder& o, int kk, int q) {
    BsPointSlots p;
    p.k = o.slot[kk];
    const int qk = q >= 0 ? (o.sorted ? o.rank[q] : q) : -1;
    p.gap = q >= 0 && o.slot[qk] != p.k + 1;
    const int4 a = o.org[p.k / BS_GROUP];
    p.O[0] = a.x; p.O[1] = a.y; p.O[2] = a.z;
    // the gap slot's group (the next group when k ends one); without a gap
    // the next slot of the same group starts the successor's own segment
    const int4 b = p.gap ? o.org[(p.k + 1) / BS_GROUP] : a;
    p.Og[0] = b.x; p.Og[1] = b.y; p.Og[2] = b.z;
    return p;
}

// The slots of one point in record block f (0: the segment si -> si + b;
// 1 + face: its image across that solid face, M(si) -> M(si) + M(b), with M
// mirroring the face-axis coordinate x -> w2 - x and the origin with it;
// the image vortex turns the other way, which the pair sum applies as the
// block's sign).  sq: the successor's position (for the gap slot).  Flags
// org[k / BS_GROUP].w when the next slot of the same group would not start
// where this segment ends (a chain that jumps by a periodic box).
__device__ __forceinline__ void bs_write_point_slots(const Grid& g, const BsOrder& o, const BsPointSlots& ps,
                                                     long long Np, int f, int face_code, const double si[3],
                                                     const double sq[3], const float b[3], bool has_seg,
                                                     float4* __restrict__ seg) {
    const int ax = f > 0 ? face_code >> 1 : -1;
    double rel[3], relq[3];
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a == ax) {
            // mirrored origin w2 - O and point w2 - x: the difference is O - x
            rel[a] = ps.O[a] - si[a];
            relq[a] = ps.Og[a] - sq[a];
            d[a] = -b[a];
        } else {
            rel[a] = min_image(g, a, si[a] - ps.O[a]);
            relq[a] = min_image(g, a, sq[a] - ps.Og[a]);
            d[a] = b[a];
        }
    }
    float val[16];
    bs_slot_values(rel, d, val);
    bs_store_slot(seg, (long long)f * Np + ps.k, val);
    if (f == 0 && has_seg && (ps.k % BS_GROUP) != BS_GROUP - 1) {
        // the next slot (same group, origin O = Og) starts at min_image(sq - O)
        bool jump = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) jump |= fabs(relq[a] - (rel[a] + (double)b[a])) > 0.5;
        if (jump) atomicOr(&o.org[ps.k / BS_GROUP].w, 1);
    }
    if (ps.gap) {
        const float z[3] = {0.f, 0.f, 0.f};
        bs_slot_values(relq, z, val);
        bs_store_slot(seg, (long long)f * Np + ps.k + 1, val);
    }
}

}  // namespace

}  // namespace vlb
