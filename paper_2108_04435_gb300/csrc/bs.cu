// Nonlocal Biot-Savart velocity of the vortex filaments (Eq. 3 of
// arXiv 2108.04435, integrated segment-wise as Sec. II.A states).
//
// For target r and straight segment s_j -> s_j + d_j, with R1 = s_j - r
// (minimum image on periodic axes) and R2 = R1 + d_j, the exact line integral
// of the Eq. 3 kernel is
//     v = kappa/(4 pi) (R1 x R2) (|R1| + |R2|) / (|R1||R2| (|R1||R2| + R1.R2)).
// The two segments touching the target are left to the local term.
//
// GB300 mapping.  This is FP32 + MUFU work (2 rsqrt + 1 reciprocal per pair),
// not a contraction, so no tensor cores.  Targets sit in registers (one or
// two per thread); source records stream through shared memory in tiles that
// one thread fetches with bulk copies (cp.async.bulk + mbarrier, double
// buffered), every lane reading each record as a broadcast.
//
// From BS_SORT_MIN points on, the points are put in a spatial (Morton) order
// once per step, and each group of BS_GROUP consecutive records stores its
// positions relative to an integer origin.  A target then meets a group
// through one offset t = (O - O_t) - h_t - l_t formed exactly once per group;
// the group's box decides, for the whole warp, between three pair paths:
//  - near (some source within BS_NEAR cells of the target in any periodic
//    image): full precision (h + l + t, the offset split in two floats), the
//    minimum image (decided in FP64 within 1e-3 of half the box, as the FP64
//    difference of the positions decides it), on-segment guard and the
//    target's own segments masked;
//  - wrap (a source may lie half a periodic box away): the same precision and
//    minimum image, no guard;
//  - far (everything else): h + t only, and the cross product R1 x d split
//    into the stored h x d and one t x (sum fac d) per group.
// Splits of the source range are summed in a fixed order (or exactly, in
// fixed point), so every result is bitwise reproducible.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>
#include <stdlib.h>

#include "eom.cuh"
#include "records.cuh"
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
    const uint32_t bytes = (uint32_t)cnt * (uint32_t)(BS_REC * sizeof(float4));
    mbar_expect_tx(bar, bytes);
    bulk_copy_g2s(dst, seg + (long long)BS_REC * jb, bytes, bar);
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

// Minimum image of r on one periodic axis (L = 0 on wall axes: unchanged).
__device__ __forceinline__ float mi_axis(float r, float L, float iL) { return fmaf(-L, round_mul_fma(r, iL), r); }

// A group whose records all lie at least BS_NEAR cells (Chebyshev) from every
// target of a warp takes the cheap pair path: the low parts are left out (an
// error of about one float ulp of the group extent and of the offset, i.e.
// ~1e-7 (1 + extent / distance) of the pair), no target can lie on a segment
// (segments are shorter than the remeshing bound, about a cell), and none of
// the target's own segments is in the group.  Measured against the FP64 sums
// of the oracle, 4 cells instead of 8 moved the relative L2 error of the
// point velocities from 1.19e-7 to 1.22e-7 on the 128x128x1024 channel
// (86k points) and from 1.71e-7 to 1.82e-7 on the sorted walled tangle
// (35k points), and made the launch 2% faster there and 8% on the 128^3 box.
constexpr float BS_NEAR = 4.f;

// One target of a Biot-Savart pass (registers of one thread): its own
// slot (origin O, parts h + l, so that the point is O + h + l) and the
// slots of the segments that belong to its local term.
struct BsTarget {
    float h[3], l[3], O[3];
    float v[3];      // sum over the sources, without the factor kappa / 4 pi
    int self, prev;  // slots of its own segment and of its predecessor's
    int excl;        // a pinned end: the image of its own segment across its wall
    int i;           // point index, -1 for an idle lane
};

// Bounding box and origin of one group of slots in shared memory.
struct BsGroup {
    float lo[3], hi[3];  // of the slots' h, relative to the origin
    float O[3];          // integer origin (exact in float)
    float sign;          // -1 for a wall-image block: the image vortex turns the other way
};

// Integer origin of the group of slot j, mirrored onto the image side for an
// image block: x_a -> w2 - x_a on the face axis a.  Returns the block index
// (0: the segments, 1 + face: their images).
struct BsImages {
    int nfaces;
    int face_code[6];
    float w2[6];         // twice the coordinate of the face
};

__device__ __forceinline__ int group_origin(const BsOrder& o, const BsImages& im, long long Np, int j, float O[3]) {
    const int f = (int)(j / Np);
    const int kk = (int)(j - (long long)f * Np);
    const int4 g = o.org[kk / BS_GROUP];
    O[0] = (float)g.x;
    O[1] = (float)g.y;
    O[2] = (float)g.z;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        if (q + 1 != f) continue;
        const int ax = im.face_code[q] >> 1;
        const float w2 = im.w2[q];
        if (ax == 0) O[0] = w2 - O[0];
        else if (ax == 1) O[1] = w2 - O[1];
        else O[2] = w2 - O[2];
    }
    return f;
}

// Target at sorted position k of N (none when k >= N), from its target
// record (four 16-byte loads).
__device__ __forceinline__ BsTarget bs_target(const BsOrder& o, int N, int k) {
    BsTarget t;
#pragma unroll
    for (int a = 0; a < 3; ++a) t.h[a] = t.l[a] = t.O[a] = t.v[a] = 0.f;
    t.self = t.prev = t.excl = -1;
    t.i = -1;
    if (k < N) {
        const float4* r = o.tgt + 4LL * k;
        const float4 a = r[0], b = r[1], c = r[2], e = r[3];
        t.h[0] = a.x; t.h[1] = a.y; t.h[2] = a.z;
        t.l[0] = a.w; t.l[1] = b.x; t.l[2] = b.y;
        t.O[0] = b.z; t.O[1] = b.w; t.O[2] = c.x;
        t.self = __float_as_int(c.y);
        t.prev = __float_as_int(c.z);
        t.excl = __float_as_int(c.w);
        t.i = __float_as_int(e.x);
    }
    return t;
}

// A 16-byte load the compiler may not move out of a loop (the target records
// are read again for every group, so that their values need no registers
// across the group's pair loop).
__device__ __forceinline__ float4 ld_reload(const float4* p) {
    float4 r;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(p));
    return r;
}

// The target of sorted position k again from its record (point index i
// already known; an idle lane, i < 0, reads nothing), with its sum zero.
__device__ __forceinline__ BsTarget bs_target_reload(const BsOrder& o, int k, int i) {
    BsTarget t;
#pragma unroll
    for (int a = 0; a < 3; ++a) t.h[a] = t.l[a] = t.O[a] = t.v[a] = 0.f;
    t.self = t.prev = t.excl = -1;
    t.i = i;
    if (i >= 0) {
        const float4* r = o.tgt + 4LL * k;
        const float4 a = ld_reload(r), b = ld_reload(r + 1), c = ld_reload(r + 2);
        t.h[0] = a.x; t.h[1] = a.y; t.h[2] = a.z;
        t.l[0] = a.w; t.l[1] = b.x; t.l[2] = b.y;
        t.O[0] = b.z; t.O[1] = b.w; t.O[2] = c.x;
        t.self = __float_as_int(c.y);
        t.prev = __float_as_int(c.z);
        t.excl = __float_as_int(c.w);
    }
    return t;
}

// The cheap pair path, along the chain of slots of one group.  Slot k's
// segment runs from its point to slot k + 1's, so with R = h + t at every
// slot (no low parts), ia = 1/|R| and rho = |R| serve the segment starting
// there and the one ending there.  For a segment from R1 to R2 = R1 + d,
// S = |R1| + |R2| and |R1||R2| + R1.R2 = (S^2 - |d|^2)/2, so the segment
// factor (|R1| + |R2|)/(|R1||R2| (|R1||R2| + R1.R2)) of Eq. 3 is
// 2 (ia1 + ia2) / (S^2 - |d|^2): one reciprocal square root per slot and one
// reciprocal per segment.  The cross product R1 x R2 = R1 x d = h x d + t x d
// is split into the slot's c = h x d and t x (sum of fac d), added once per
// group.  A pair p (slots p and p + 32) is evaluated packed (FP32x2), so the
// group's two halves walk their chains side by side.

// ia and rho at the two slots of pair p, for each target offset t, and the
// pair's |d|^2 for its segments.  |R|^2 = |h + t|^2 is formed as
// (|h|^2 + |t|^2) + 2 h.t with |h|^2 from the slot and 2t, |t|^2 per group
// (t2, tt: held in both halves of a float2): three fused multiply-adds and
// an add instead of three adds and three multiply-adds.  The group origin
// sits at the centre of the group's box, so |h| is at most about half its
// extent, and the cancellation of |t|^2 against 2 h.t costs about
// (|h| + |R|)^2 / |R|^2 float ulps of |R|^2 at the far path's distance of 4
// cells or more (measured: the point velocities of the 86k-point channel
// move from 1.19e-7 to 1.22e-7 of the FP64 sums when the far path starts at
// 4 cells instead of 8).
template <int TGT>
__device__ __forceinline__ void chain_head(const float4* __restrict__ Q, const float2 (&t2)[TGT][3],
                                           const float2 (&tt)[TGT], float2 (&ia)[TGT], float2 (&rho)[TGT],
                                           float2& dd) {
    const float4 q0 = Q[0], q1 = Q[1], q8 = Q[8];
    const float2 hx = make_float2(q0.x, q0.y), hy = make_float2(q0.z, q0.w), hz = make_float2(q1.x, q1.y);
    const float2 hh = make_float2(q8.x, q8.y);
    dd = make_float2(q1.z, q1.w);
#pragma unroll
    for (int u = 0; u < TGT; ++u) {
        const float2 a2 =
            __ffma2_rn(hz, t2[u][2], __ffma2_rn(hy, t2[u][1], __ffma2_rn(hx, t2[u][0], __fadd2_rn(hh, tt[u]))));
        ia[u] = make_float2(rsqrt_approx(a2.x), rsqrt_approx(a2.y));
        rho[u] = __fmul2_rn(a2, ia[u]);
    }
}

// The segments of the slots of pair p (|d|^2 from its head), from (ia0,
// rho0) at their starts to (ia1, rho1) at their ends, into the sums of fac c
// and fac d (fac halved).
template <int TGT>
__device__ __forceinline__ void chain_segments(const float4* __restrict__ Q, const float2& dd,
                                               const float2 (&ia0)[TGT], const float2 (&rho0)[TGT],
                                               const float2 (&ia1)[TGT], const float2 (&rho1)[TGT],
                                               float2 (&av)[TGT][3], float2 (&aw)[TGT][3]) {
    const float4 q2 = Q[2], q3 = Q[3], q4 = Q[4];
    const float2 mdd = make_float2(-dd.x, -dd.y);
    const float2 dx = make_float2(q2.x, q2.y), dy = make_float2(q2.z, q2.w), dz = make_float2(q3.x, q3.y);
    const float2 cx = make_float2(q3.z, q3.w), cy = make_float2(q4.x, q4.y), cz = make_float2(q4.z, q4.w);
#pragma unroll
    for (int u = 0; u < TGT; ++u) {
        const float2 S = __fadd2_rn(rho0[u], rho1[u]);
        const float2 den = __ffma2_rn(S, S, mdd);
        const float2 fac = __fmul2_rn(__fadd2_rn(ia0[u], ia1[u]), make_float2(rcp_approx(den.x), rcp_approx(den.y)));
        av[u][0] = __ffma2_rn(fac, cx, av[u][0]);
        av[u][1] = __ffma2_rn(fac, cy, av[u][1]);
        av[u][2] = __ffma2_rn(fac, cz, av[u][2]);
        aw[u][0] = __ffma2_rn(fac, dx, aw[u][0]);
        aw[u][1] = __ffma2_rn(fac, dy, aw[u][1]);
        aw[u][2] = __ffma2_rn(fac, dz, aw[u][2]);
    }
}

// The chain of one group for TGT targets at offsets t: pair p's segments end
// at pair p + 1's slots, except slot 31's, which ends at slot 32 (the first
// pair's other half), and slot 63's, which ends at the end point its record
// stores (the next slot is in another group).  Returns the sums of fac c
// and fac d with fac halved.
template <int TGT>
__device__ __forceinline__ void chain_group(const float4* __restrict__ T, const float (&th)[TGT][3],
                                            float2 (&av)[TGT][3], float2 (&aw)[TGT][3]) {
    float2 t[TGT][3], tt[TGT];
#pragma unroll
    for (int u = 0; u < TGT; ++u) {
#pragma unroll
        for (int a = 0; a < 3; ++a) t[u][a] = make_float2(2.f * th[u][a], 2.f * th[u][a]);
        const float q = fmaf(th[u][0], th[u][0], fmaf(th[u][1], th[u][1], th[u][2] * th[u][2]));
        tt[u] = make_float2(q, q);
    }
    // the end of the group: slot 31 ends at slot 32, slot 63 at its stored end point
    auto last_end = [&](float2 (&ia1)[TGT], float2 (&rho1)[TGT], float ia32[TGT], float rho32[TGT]) {
        const float4* Q = T + BS_PAIR * (BS_GROUP / 2 - 1);
        const float4 q6 = Q[6], q7 = Q[7];  // values 13-15 (slot 63 in the .y halves)
#pragma unroll
        for (int u = 0; u < TGT; ++u) {
            const float ex = q6.w + th[u][0], ey = q7.y + th[u][1], ez = q7.w + th[u][2];
            const float b2 = ex * ex + ey * ey + ez * ez;
            const float ib = rsqrt_approx(b2);
            ia1[u] = make_float2(ia32[u], ib);
            rho1[u] = make_float2(rho32[u], b2 * ib);
        }
    };
    float2 ia0[TGT], rho0[TGT], dd0;
    chain_head<TGT>(T, t, tt, ia0, rho0, dd0);
    float ia32[TGT], rho32[TGT];
#pragma unroll
    for (int u = 0; u < TGT; ++u) {
        ia32[u] = ia0[u].y;
        rho32[u] = rho0[u].y;
    }
#pragma unroll 2
    for (int p = 0; p < BS_GROUP / 2 - 1; ++p) {
        float2 ia1[TGT], rho1[TGT], dd1;
        chain_head<TGT>(T + BS_PAIR * (p + 1), t, tt, ia1, rho1, dd1);
        chain_segments<TGT>(T + BS_PAIR * p, dd0, ia0, rho0, ia1, rho1, av, aw);
#pragma unroll
        for (int u = 0; u < TGT; ++u) {
            ia0[u] = ia1[u];
            rho0[u] = rho1[u];
        }
        dd0 = dd1;
    }
    float2 ia1[TGT], rho1[TGT];
    last_end(ia1, rho1, ia32, rho32);
    chain_segments<TGT>(T + BS_PAIR * (BS_GROUP / 2 - 1), dd0, ia0, rho0, ia1, rho1, av, aw);
}

// Minimum image of one component of R1 on a periodic axis (L = 0 on wall
// axes: unchanged).  r = (h + t_hi) + (l + t_lo) carries FP32 rounding, so
// within 1e-3 of half the box it cannot tell which image is nearer.  There
// the image is chosen from the exact sum x = s + c, s = fl(h + t_hi) and c
// its TwoSum error plus l + t_lo (exact to ~1e-13 cells): y0 = s - kL is
// exact (Sterbenz), and so is y0 -/+ L/2, so the sign of (y0 -/+ L/2) + c,
// which decides the image, is the sign an FP64 evaluation of s_j - r gives.
__device__ __forceinline__ float mi_exact(float r, float h, float th, float l, float tl, float L, float iL) {
    const float rm = mi_axis(r, L, iL);
    if (fabsf(rm) > 0.5f * L - 1e-3f && L > 0.f) {
        const float s = __fadd_rn(h, th), bb = __fsub_rn(s, h);
        const float c = __fadd_rn(__fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(th, bb)), __fadd_rn(l, tl));
        const float y0 = __fsub_rn(s, __fmul_rn(L, rintf(__fmul_rn(s, iL))));
        const float hl = 0.5f * L;
        float y = __fadd_rn(y0, c);
        if (__fadd_rn(__fsub_rn(y0, hl), c) > 0.f) y = __fsub_rn(y, L);
        else if (__fadd_rn(__fadd_rn(y0, hl), c) < 0.f) y = __fadd_rn(y, L);
        return y;
    }
    return rm;
}

// Pair paths with R1 in full precision: R1 = (h + t_hi) + (l + t_lo), the
// minimum image on periodic axes.  GUARD (near groups): the on-segment guard
// and the target's own segments (left to the local term) masked out by
// slot number j.  Without GUARD (groups some target sees across half a
// periodic box, none near): neither can occur.
template <bool PERIODIC, bool GUARD>
__device__ __forceinline__ void pair_precise(float hx, float hy, float hz, float dd, float dx, float dy, float dz,
                                             float lx, float ly, float lz, int j, const float th[3],
                                             const float tl[3], const BsTarget& t, float v[3], const BoxF& box,
                                             float sign) {
    float r1x = (hx + th[0]) + (lx + tl[0]);
    float r1y = (hy + th[1]) + (ly + tl[1]);
    float r1z = (hz + th[2]) + (lz + tl[2]);
    if (PERIODIC) {
        if (sign > 0.f) {
            r1x = mi_exact(r1x, hx, th[0], lx, tl[0], box.Lx, box.iLx);
            r1y = mi_exact(r1y, hy, th[1], ly, tl[1], box.Ly, box.iLy);
            r1z = mi_exact(r1z, hz, th[2], lz, tl[2], box.Lz, box.iLz);
        } else {
            // a wall image runs from M(s_q) to M(s_i) (its slot stores it the
            // other way round): its periodic image is that of M(s_q), the
            // slot's end point (decided in FP32)
            r1x = fmaf(-box.Lx, round_mul_fma(r1x + dx, box.iLx), r1x);
            r1y = fmaf(-box.Ly, round_mul_fma(r1y + dy, box.iLy), r1y);
            r1z = fmaf(-box.Lz, round_mul_fma(r1z + dz, box.iLz), r1z);
        }
    }
    const float a2 = r1x * r1x + r1y * r1y + r1z * r1z;
    const float rd = r1x * dx + r1y * dy + r1z * dz;
    const float b2 = fmaf(2.f, rd, a2) + dd;
    const float ia = rsqrt_approx(a2), ib = rsqrt_approx(b2);
    const float P = ia * ib;
    const float cx = r1y * dz - r1z * dy, cy = r1z * dx - r1x * dz, cz = r1x * dy - r1y * dx;
    // The factor's denominator e = |R1||R2| + R1.R2 (over |R1||R2|: 1 + P R1.R2)
    // cancels when the target lies near the segment between its ends
    // (R1.R2 < 0, the angle between R1 and R2 near pi).  There it is formed as
    // |R1 x d|^2 / (|R1||R2| - R1.R2), exactly equal and free of
    // cancellation: fac = (ia + ib)(1 - P R1.R2) / (P |R1 x d|^2).
    const float s12 = a2 + rd;
    const float cr2 = fmaf(cz, cz, fmaf(cy, cy, cx * cx));
    const bool anti = s12 < 0.f;
    const float num = (ia + ib) * (anti ? fmaf(-P, s12, 1.f) : P);
    const float dn = anti ? P * cr2 : fmaf(P, s12, 1.f);
    const float fac = num * rcp_approx(dn) * sign;
    float c = fac;
    if (GUARD) {
        // 1 + P R1.R2 <= 1e-6: the target lies on the segment (or coincides
        // with an end point), where the integral is not defined; NaN and
        // infinity fail too.  Slots without a segment (gap and padding slots,
        // a line's last point) are skipped: a gap slot may hold the target's
        // own point, ~1e-14 away in another group's origin, where fac
        // overflows and fac * 0 would be NaN.
        const bool on = anti ? !(P * dn > 1e-6f * fmaf(-P, s12, 1.f)) : !(dn > 1e-6f);
        const bool use = (dd > 0.f) & !on & (dn < 3.0e38f) & (fabsf(fac) < 3.0e38f) & (j != t.self) &
                         (j != t.prev) & (j != t.excl);
        c = use ? fac : 0.f;
    }
    v[0] = fmaf(c, cx, v[0]);
    v[1] = fmaf(c, cy, v[1]);
    v[2] = fmaf(c, cz, v[2]);
}

// Both slots of a pair on the precise path (q0..q6: values 0-13 of both);
// j is the first slot, j + 32 the second, Np the slots of a block (the
// image blocks, j >= Np, turn the other way).
template <bool PERIODIC, bool GUARD, int TGT>
__device__ __forceinline__ void pair2_precise(const float4* __restrict__ Q, int j, const float (&th)[TGT][3],
                                              const float (&tl)[TGT][3], BsTarget (&t)[TGT], const BoxF& box,
                                              int Np) {
    const float4 q0 = Q[0], q1 = Q[1], q2 = Q[2], q3 = Q[3], q5 = Q[5], q6 = Q[6];
    const float sign = j >= Np ? -1.f : 1.f;
#pragma unroll
    for (int u = 0; u < TGT; ++u) {
        pair_precise<PERIODIC, GUARD>(q0.x, q0.z, q1.x, q1.z, q2.x, q2.z, q3.x, q5.x, q5.z, q6.x, j, th[u], tl[u], t[u],
                                      t[u].v, box, sign);
        pair_precise<PERIODIC, GUARD>(q0.y, q0.w, q1.y, q1.w, q2.y, q2.w, q3.y, q5.y, q5.w, q6.y, j + BS_GROUP / 2,
                                      th[u], tl[u], t[u], t[u].v, box, sign);
    }
}

__device__ __forceinline__ float2 fsub2(float2 x, float2 y) { return __fadd2_rn(x, make_float2(-y.x, -y.y)); }

// The wrap path for the two slots of pair p (groups that no target of the
// warp sees within BS_NEAR cells, but some of whose sources may lie half a
// periodic box away): R1 = h + t without the low parts, as on the far path,
// and the minimum image of every pair decided in FP32 (for a wall-image slot,
// that of its end point, reading 21) on the axes `axes` where the group may
// reach half a box from some target of the warp (on the others every source
// already lies within half a box, in the group's image).  When some lane finds a pair within
// 1e-3 cells of half the box, where dropping the low parts could change the
// decision, the warp takes that pair on the precise path instead, which
// decides it exactly.  Adds the pair's sums into v (the block's sign
// applied by the caller).
template <int TGT>
__device__ __forceinline__ void pair2_wrap(const float4* __restrict__ Q, int j, const float (&th)[TGT][3],
                                           const float (&tl)[TGT][3], BsTarget (&t)[TGT], const BoxF& box,
                                           int Np, int axes, float2 (&v)[TGT][3]) {
    const float4 q0 = Q[0], q1 = Q[1], q2 = Q[2], q3 = Q[3];
    const float2 hx = make_float2(q0.x, q0.y), hy = make_float2(q0.z, q0.w), hz = make_float2(q1.x, q1.y);
    const float2 dd = make_float2(q1.z, q1.w);
    const float2 dx = make_float2(q2.x, q2.y), dy = make_float2(q2.z, q2.w), dz = make_float2(q3.x, q3.y);
    const bool img = j >= Np;
    const float2 ex = img ? dx : make_float2(0.f, 0.f), ey = img ? dy : make_float2(0.f, 0.f),
                 ez = img ? dz : make_float2(0.f, 0.f);
    const float M = 12582912.0f;  // 1.5 * 2^23: adding it rounds to the nearest integer
    float2 r[TGT][3];
    bool tie = false;
#pragma unroll
    for (int u = 0; u < TGT; ++u) {
        r[u][0] = __fadd2_rn(hx, make_float2(th[u][0], th[u][0]));
        r[u][1] = __fadd2_rn(hy, make_float2(th[u][1], th[u][1]));
        r[u][2] = __fadd2_rn(hz, make_float2(th[u][2], th[u][2]));
        const float2 e[3] = {ex, ey, ez};
        const float L[3] = {box.Lx, box.Ly, box.Lz}, iL[3] = {box.iLx, box.iLy, box.iLz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if ((axes >> a) & 1) {
                const float2 z = __fadd2_rn(r[u][a], e[a]);
                const float2 k = fsub2(__ffma2_rn(z, make_float2(iL[a], iL[a]), make_float2(M, M)),
                                            make_float2(M, M));
                r[u][a] = __ffma2_rn(make_float2(-L[a], -L[a]), k, r[u][a]);
                const float2 w = __fadd2_rn(r[u][a], e[a]);
                tie |= (fabsf(w.x) > 0.5f * L[a] - 1e-3f) | (fabsf(w.y) > 0.5f * L[a] - 1e-3f);
            }
        }
    }
    if (__any_sync(0xffffffffu, tie)) {
        pair2_precise<true, false, TGT>(Q, j, th, tl, t, box, Np);
        return;
    }
#pragma unroll
    for (int u = 0; u < TGT; ++u) {
        const float2 rx = r[u][0], ry = r[u][1], rz = r[u][2];
        const float2 a2 = __ffma2_rn(rz, rz, __ffma2_rn(ry, ry, __fmul2_rn(rx, rx)));
        const float2 rd = __ffma2_rn(rz, dz, __ffma2_rn(ry, dy, __fmul2_rn(rx, dx)));
        const float2 b2 = __fadd2_rn(__ffma2_rn(make_float2(2.f, 2.f), rd, a2), dd);
        const float2 ia = make_float2(rsqrt_approx(a2.x), rsqrt_approx(a2.y));
        const float2 ib = make_float2(rsqrt_approx(b2.x), rsqrt_approx(b2.y));
        const float2 P = __fmul2_rn(ia, ib);
        const float2 den = __ffma2_rn(P, __fadd2_rn(a2, rd), make_float2(1.f, 1.f));
        const float2 fac = __fmul2_rn(__fmul2_rn(__fadd2_rn(ia, ib), P), make_float2(rcp_approx(den.x), rcp_approx(den.y)));
        v[u][0] = __ffma2_rn(fac, fsub2(__fmul2_rn(ry, dz), __fmul2_rn(rz, dy)), v[u][0]);
        v[u][1] = __ffma2_rn(fac, fsub2(__fmul2_rn(rz, dx), __fmul2_rn(rx, dz)), v[u][1]);
        v[u][2] = __ffma2_rn(fac, fsub2(__fmul2_rn(rx, dy), __fmul2_rn(ry, dx)), v[u][2]);
    }
}

// The near path for the two slots of pair p, packed: the arithmetic of
// pair_precise (low parts, minimum image on periodic axes, the on-segment
// and own-segment guard, the cancellation-free denominator) on both slots at
// once in FP32x2, into the sums v (the block's sign applied by the caller).
// Where some lane's minimum image falls within 1e-3 of half the box, the
// warp takes this pair on the scalar precise path, which decides the image
// from the exact float-float sum of the parts.
template <bool PERIODIC, int TGT>
__device__ __forceinline__ void pair2_near(const float4* __restrict__ Q, int j, const float (&th)[TGT][3],
                                           const float (&tl)[TGT][3], BsTarget (&t)[TGT], const BoxF& box,
                                           int Np, float2 (&v)[TGT][3]) {
    const float4 q0 = Q[0], q1 = Q[1], q2 = Q[2], q3 = Q[3], q5 = Q[5], q6 = Q[6];
    const float2 hh[3] = {make_float2(q0.x, q0.y), make_float2(q0.z, q0.w), make_float2(q1.x, q1.y)};
    const float2 ll[3] = {make_float2(q5.x, q5.y), make_float2(q5.z, q5.w), make_float2(q6.x, q6.y)};
    const float2 dd = make_float2(q1.z, q1.w);
    const float2 dx = make_float2(q2.x, q2.y), dy = make_float2(q2.z, q2.w), dz = make_float2(q3.x, q3.y);
    const float2 dv[3] = {dx, dy, dz};
    const bool img = j >= Np;
    const float L[3] = {box.Lx, box.Ly, box.Lz}, iL[3] = {box.iLx, box.iLy, box.iLz};
    const float2 M2 = make_float2(12582912.0f, 12582912.0f);  // 1.5 * 2^23: adding it rounds to an integer
    float2 r[TGT][3];
    bool tie = false;
#pragma unroll
    for (int u = 0; u < TGT; ++u)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            r[u][a] = __fadd2_rn(__fadd2_rn(hh[a], make_float2(th[u][a], th[u][a])),
                                 __fadd2_rn(ll[a], make_float2(tl[u][a], tl[u][a])));
            if (PERIODIC) {
                const float2 z = img ? __fadd2_rn(r[u][a], dv[a]) : r[u][a];
                const float2 k = fsub2(__ffma2_rn(z, make_float2(iL[a], iL[a]), M2), M2);
                r[u][a] = __ffma2_rn(make_float2(-L[a], -L[a]), k, r[u][a]);
                if (!img)
                    tie |= (L[a] > 0.f) & ((fabsf(r[u][a].x) > 0.5f * L[a] - 1e-3f) |
                                           (fabsf(r[u][a].y) > 0.5f * L[a] - 1e-3f));
            }
        }
    if (PERIODIC && __any_sync(0xffffffffu, tie)) {
        pair2_precise<PERIODIC, true, TGT>(Q, j, th, tl, t, box, Np);
        return;
    }
    const float2 one = make_float2(1.f, 1.f);
#pragma unroll
    for (int u = 0; u < TGT; ++u) {
        const float2 rx = r[u][0], ry = r[u][1], rz = r[u][2];
        const float2 a2 = __ffma2_rn(rz, rz, __ffma2_rn(ry, ry, __fmul2_rn(rx, rx)));
        const float2 rd = __ffma2_rn(rz, dz, __ffma2_rn(ry, dy, __fmul2_rn(rx, dx)));
        const float2 b2 = __fadd2_rn(__ffma2_rn(make_float2(2.f, 2.f), rd, a2), dd);
        const float2 ia = make_float2(rsqrt_approx(a2.x), rsqrt_approx(a2.y));
        const float2 ib = make_float2(rsqrt_approx(b2.x), rsqrt_approx(b2.y));
        const float2 P = __fmul2_rn(ia, ib);
        const float2 cx = fsub2(__fmul2_rn(ry, dz), __fmul2_rn(rz, dy));
        const float2 cy = fsub2(__fmul2_rn(rz, dx), __fmul2_rn(rx, dz));
        const float2 cz = fsub2(__fmul2_rn(rx, dy), __fmul2_rn(ry, dx));
        // the denominator as in pair_precise: 1 + P R1.R2, or where R1.R2 < 0
        // P |R1 x d|^2 over 1 - P R1.R2 (exactly equal, free of cancellation)
        const float2 s12 = __fadd2_rn(a2, rd);
        const float2 cr2 = __ffma2_rn(cz, cz, __ffma2_rn(cy, cy, __fmul2_rn(cx, cx)));
        const float2 alt = __ffma2_rn(make_float2(-P.x, -P.y), s12, one);
        const float2 pos = __ffma2_rn(P, s12, one);
        const float2 pcr = __fmul2_rn(P, cr2);
        const bool ax = s12.x < 0.f, ay = s12.y < 0.f;
        const float2 num = __fmul2_rn(__fadd2_rn(ia, ib), make_float2(ax ? alt.x : P.x, ay ? alt.y : P.y));
        const float2 dn = make_float2(ax ? pcr.x : pos.x, ay ? pcr.y : pos.y);
        const float2 fac = __fmul2_rn(num, make_float2(rcp_approx(dn.x), rcp_approx(dn.y)));
        const float2 pdn = __fmul2_rn(P, dn);
        // the guard of pair_precise, lane by lane
        const bool onx = ax ? !(pdn.x > 1e-6f * alt.x) : !(dn.x > 1e-6f);
        const bool ony = ay ? !(pdn.y > 1e-6f * alt.y) : !(dn.y > 1e-6f);
        const int j1 = j + BS_GROUP / 2;
        const bool ux = (dd.x > 0.f) & !onx & (dn.x < 3.0e38f) & (fabsf(fac.x) < 3.0e38f) & (j != t[u].self) &
                        (j != t[u].prev) & (j != t[u].excl);
        const bool uy = (dd.y > 0.f) & !ony & (dn.y < 3.0e38f) & (fabsf(fac.y) < 3.0e38f) & (j1 != t[u].self) &
                        (j1 != t[u].prev) & (j1 != t[u].excl);
        const float2 c = make_float2(ux ? fac.x : 0.f, uy ? fac.y : 0.f);
        v[u][0] = __ffma2_rn(c, cx, v[u][0]);
        v[u][1] = __ffma2_rn(c, cy, v[u][1]);
        v[u][2] = __ffma2_rn(c, cz, v[u][2]);
    }
}

// Offset of a group (origin O, record box [lo, hi]) from a target: the
// integer part D = O - O_t is exact, and on periodic axes D is moved by a
// whole box so that the group's centre is the nearest image.  Returns
// t_hi = fl(D - h_t) and flags whether the group may hold a source within
// BS_NEAR of the target (near) and whether some source may lie more than half
// a box away on a periodic axis in that image (wrap).
template <bool PERIODIC>
__device__ __forceinline__ void group_offset(const BsGroup& G, const BsTarget& t, const BoxF& box, float D[3],
                                             float th[3], bool& near, int& wrap) {
    const float L[3] = {box.Lx, box.Ly, box.Lz}, iL[3] = {box.iLx, box.iLy, box.iLz};
    float dist = 0.f;
    wrap = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        D[a] = G.O[a] - t.O[a];
        if (PERIODIC) D[a] -= L[a] * rintf((D[a] + 0.5f * (G.lo[a] + G.hi[a]) - t.h[a]) * iL[a]);
        th[a] = D[a] - t.h[a];
        const float lo = th[a] + G.lo[a], hi = th[a] + G.hi[a];
        float da = fmaxf(fmaxf(lo, -hi), 0.f);
        if (PERIODIC) {
            // the box's neighbouring images may come closer (L = 0 on wall axes: the same box)
            da = fminf(da, fmaxf(fmaxf(lo - L[a], L[a] - hi), 0.f));
            da = fminf(da, fmaxf(fmaxf(lo + L[a], -(hi + L[a])), 0.f));
            if ((L[a] > 0.f) & ((hi > 0.5f * L[a] - 0.01f) | (lo < 0.01f - 0.5f * L[a]))) wrap |= 1 << a;
        }
        dist = fmaxf(dist, da);
    }
    near = dist < BS_NEAR;
}

// Shared-memory stages of the source pipeline.  Every tile of BS_TILE
// records lands by one bulk copy that completes full[b]; the warps consume
// it independently (a warp's groups may take another pair path than its
// neighbours' and so take longer), and the warp that releases the buffer
// last (a counter per stage) issues the copy of the tile BS_STAGES further
// on.  No block-wide barrier is needed per tile, so warps can drift up to
// that many tiles apart.  One target per thread: three stages, so that eight
// blocks fit on an SM; two targets: four.
template <int TGT>
__host__ __device__ constexpr int bs_stages() { return TGT == 1 ? 3 : 4; }

struct BsSmem {
    int nst;          // stages in use
    float4 (*tile)[BS_TILE * BS_REC];
    uint64_t* full;   // [nst] completed by the copy's byte count
    int* release;     // [nst] warps done with the stage's current tile
    int* fills;       // [nst] copies issued into the stage so far
    int* s_item;
    int* s_last;
    int* s_abort;     // a wait timed out: every warp leaves the pass
};

__device__ __forceinline__ void bs_smem_init(const BsSmem& sm) {
    if (threadIdx.x < sm.nst) {
        sm.release[threadIdx.x] = 0;
        sm.fills[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) {
        for (int b = 0; b < sm.nst; ++b) mbar_init(&sm.full[b], 1);
        *sm.s_abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
}

// Copy tile number `tile` of the range [j0, j1) into the stage of the
// block's tile sequence number q.
__device__ __forceinline__ void bs_fill(const BsSmem& sm, const float4* seg, uint32_t q, int j0, int j1, int tile) {
    const int b = (int)(q % (uint32_t)sm.nst);
    const int jb = j0 + tile * BS_TILE;
    sm.fills[b] += 1;
    issue_tile(sm.tile[b], seg, jb, min(BS_TILE, j1 - jb), &sm.full[b]);
}

// Box, origin and sign of one group of slots.  The box was stored by the
// stage geometry in values 13-15 of slots 0 and 1 (the x halves of pairs 0
// and 1); a group whose chain jumps by a periodic box has an unbounded one,
// which sends it to the full-precision path (as a near group).
__device__ __forceinline__ BsGroup group_box(const float4* __restrict__ T, int j, const BsOrder& o,
                                             const BsImages& im, long long Np) {
    BsGroup G;
    const float4 a6 = T[6], a7 = T[7], b6 = T[BS_PAIR + 6], b7 = T[BS_PAIR + 7];
    G.lo[0] = a6.z; G.lo[1] = a7.x; G.lo[2] = a7.z;
    G.hi[0] = b6.z; G.hi[1] = b7.x; G.hi[2] = b7.z;
    G.sign = group_origin(o, im, Np, j, G.O) > 0 ? -1.f : 1.f;
    return G;
}

// The sums of one group of slots (slot numbers gbase ..) for TGT targets per
// thread (sorted positions kbase ..), on the path the warp's targets need,
// added into acc[].v.  The targets' positions and slots are read again from
// their records here rather than kept in registers across groups.
template <bool PERIODIC, int TGT>
__device__ __forceinline__ void bs_group(const float4* __restrict__ T, int gbase, const BsGroup& G,
                                         BsTarget (&acc)[TGT], const BsOrder& o, int kbase, const BoxF& box,
                                         int Np) {
    BsTarget t[TGT];
#pragma unroll
    for (int u = 0; u < TGT; ++u) t[u] = bs_target_reload(o, kbase + u, acc[u].i);
    float D[TGT][3], th[TGT][3];
    bool nearL = false;
    int wrapL = 0;
#pragma unroll
    for (int u = 0; u < TGT; ++u) {
        bool nu;
        int wu;
        group_offset<PERIODIC>(G, t[u], box, D[u], th[u], nu, wu);
        const bool own = (unsigned)(t[u].self - gbase) < (unsigned)BS_GROUP ||
                         (unsigned)(t[u].prev - gbase) < (unsigned)BS_GROUP ||
                         (unsigned)(t[u].excl - gbase) < (unsigned)BS_GROUP;
        if (t[u].i >= 0) {
            nearL |= nu | own;
            wrapL |= wu;
        }
    }
    const bool nearW = __any_sync(0xffffffffu, nearL);
    // periodic axes on which some source may lie half a box away for some lane
    const int wrapW = PERIODIC ? (int)__reduce_or_sync(0xffffffffu, (unsigned)wrapL) : 0;
    if (nearW || wrapW) {
        // low part of the offset: t = D - h_t - l_t with D - h_t split exactly (TwoSum)
        float tl[TGT][3];
#pragma unroll
        for (int u = 0; u < TGT; ++u)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float s = th[u][a], x = D[u][a], y = -t[u].h[a];
                const float bb = s - x;
                tl[u][a] = ((x - (s - bb)) + (y - bb)) - t[u].l[a];
            }
        // two pairs per pass with one target per thread: with few points the
        // kernel is latency-bound, and the pairs are independent chains
        if (nearW) {
            float2 v[TGT][3];
#pragma unroll
            for (int u = 0; u < TGT; ++u)
#pragma unroll
                for (int a = 0; a < 3; ++a) v[u][a] = make_float2(0.f, 0.f);
            for (int p = 0; p < BS_GROUP / 2; ++p) pair2_near<PERIODIC, TGT>(T + BS_PAIR * p, gbase + p, th, tl, t, box, Np, v);
#pragma unroll
            for (int u = 0; u < TGT; ++u)
#pragma unroll
                for (int a = 0; a < 3; ++a) t[u].v[a] = fmaf(G.sign, v[u][a].x + v[u][a].y, t[u].v[a]);
        } else if (PERIODIC) {
            float2 v[TGT][3];
#pragma unroll
            for (int u = 0; u < TGT; ++u)
#pragma unroll
                for (int a = 0; a < 3; ++a) v[u][a] = make_float2(0.f, 0.f);
#pragma unroll 2
            for (int p = 0; p < BS_GROUP / 2; ++p)
                pair2_wrap<TGT>(T + BS_PAIR * p, gbase + p, th, tl, t, box, Np, wrapW, v);
#pragma unroll
            for (int u = 0; u < TGT; ++u)
#pragma unroll
                for (int a = 0; a < 3; ++a) t[u].v[a] = fmaf(G.sign, v[u][a].x + v[u][a].y, t[u].v[a]);
        }
    } else {
        float2 av[TGT][3], aw[TGT][3];
#pragma unroll
        for (int u = 0; u < TGT; ++u)
#pragma unroll
            for (int a = 0; a < 3; ++a) av[u][a] = aw[u][a] = make_float2(0.f, 0.f);
        chain_group<TGT>(T, th, av, aw);
        // the factor 2 of the halved segment factor, and the block's sign
        const float sc = 2.f * G.sign;
#pragma unroll
        for (int u = 0; u < TGT; ++u) {
            const float wx = aw[u][0].x + aw[u][0].y, wy = aw[u][1].x + aw[u][1].y, wz = aw[u][2].x + aw[u][2].y;
            t[u].v[0] = fmaf(sc, (av[u][0].x + av[u][0].y) + (th[u][1] * wz - th[u][2] * wy), t[u].v[0]);
            t[u].v[1] = fmaf(sc, (av[u][1].x + av[u][1].y) + (th[u][2] * wx - th[u][0] * wz), t[u].v[1]);
            t[u].v[2] = fmaf(sc, (av[u][2].x + av[u][2].y) + (th[u][0] * wy - th[u][1] * wx), t[u].v[2]);
        }
    }
#pragma unroll
    for (int u = 0; u < TGT; ++u)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[u].v[a] += t[u].v[a];
}

// Work items are (target tile of BS_TPB * TGT points, source split).  Block b
// starts with item b and takes further items from a device counter (reset by
// the stage-geometry kernel), so the grid is fixed and no item depends on a
// host-side estimate of N.  With several splits, each item stores its partial
// sums and the last item of a target tile adds them in split order (fixed,
// hence deterministic) into vel; with one split the item writes vel directly.
// `q` counts the tiles the block has consumed across items (stage q %
// stages, fill phase (q / stages) & 1).  A thread's TGT targets are
// consecutive sorted positions, so that a warp's targets are as compact as
// the order makes them.  Returns false after a timed-out tile copy (status
// TIMEOUT set).
template <bool PERIODIC, int TGT, bool EOM, bool ACC>
__device__ bool bs_work(const float4* __restrict__ seg, const int* __restrict__ prev, int* __restrict__ counters,
                        int* __restrict__ tile_ticket, int cap, const BoxF& box, float kq, float* __restrict__ part,
                        float* __restrict__ vel, const EomArgs& ea, const BsImages& im, const BsOrder& o, int nsm,
                        const BsSmem& sm, uint32_t& q, long long* __restrict__ vacc) {
    int& s_item = *sm.s_item;
    int& s_last = *sm.s_last;
    volatile int* s_abort = sm.s_abort;
    constexpr int TT = BS_TPB * TGT;  // targets per item
    constexpr int NW = BS_TPB / 32;   // warps per block
    constexpr uint32_t NST = bs_stages<TGT>();
    const int lane = threadIdx.x & 31;
    const int N = counters[CNT_N];
    if (N <= 0) return true;
    const long long Np = bs_block(counters[CNT_NSLOT]);
    const int nsrc = (int)(Np * (1 + im.nfaces));  // segments, then their wall images
    const int ns = bs_splits(N, TT, nsm, nsrc / BS_GROUP);
    const int ntb = (N + TT - 1) / TT;
    const int nitems = ntb * ns;
    // splits start on group boundaries, so that every tile starts on one
    const int chunk = (nsrc / BS_GROUP + ns - 1) / ns * BS_GROUP;
    if ((int)blockIdx.x >= nitems) return true;
    int item = blockIdx.x;
    while (true) {
        const int tb = item % ntb, split = item / ntb;
        const int j0 = min(nsrc, split * chunk);
        const int j1 = min(nsrc, j0 + chunk);
        const int ntiles = j1 > j0 ? (j1 - j0 + BS_TILE - 1) / BS_TILE : 0;
        // every stage is free here (the item before ended with a block barrier)
        if (threadIdx.x == 0)
            for (int k = 0; k < min(NST, ntiles); ++k) bs_fill(sm, seg, q + (uint32_t)k, j0, j1, k);
        BsTarget t[TGT];
#pragma unroll
        for (int u = 0; u < TGT; ++u) t[u] = bs_target(o, N, tb * TT + threadIdx.x * TGT + u);
        for (int tt = 0; tt < ntiles; ++tt) {
            const uint32_t qt = q + (uint32_t)tt;
            const int b = (int)(qt % NST);
            if (*s_abort) break;
            if (!mbar_wait_bounded(&sm.full[b], (qt / NST) & 1u)) {
                if (lane == 0) {
                    *s_abort = 1;
                    atomicOr(&counters[CNT_STATUS], ST_TIMEOUT);
                }
                break;
            }
            const int jb = j0 + tt * BS_TILE;
            const int cnt = min(BS_TILE, j1 - jb);
            const float4* T = sm.tile[b];
#pragma unroll 1
            for (int gi = 0; gi * BS_GROUP < cnt; ++gi) {
                const BsGroup G = group_box(T + BS_REC * BS_GROUP * gi, jb + gi * BS_GROUP, o, im, Np);
                bs_group<PERIODIC, TGT>(T + BS_REC * BS_GROUP * gi, jb + gi * BS_GROUP, G, t, o,
                                        tb * TT + threadIdx.x * TGT, box, (int)Np);
            }
            // release the stage; the last warp out refills it with the tile NST on
            __syncwarp();
            if (lane == 0 && atomicAdd(&sm.release[b], 1) == NW - 1) {
                sm.release[b] = 0;
                if (tt + NST < ntiles) bs_fill(sm, seg, qt + NST, j0, j1, tt + NST);
            }
        }
        q += (uint32_t)ntiles;
        if (__syncthreads_or(*s_abort)) return false;
#pragma unroll
        for (int v = 0; v < TGT; ++v)
#pragma unroll
            for (int a = 0; a < 3; ++a) t[v].v[a] *= kq;
        if (ACC) {
            // ACC: each split adds its sums in fixed point (exact, in any
            // order); the equation-of-motion kernel that follows reads them
#pragma unroll
            for (int v = 0; v < TGT; ++v) {
                const int i = t[v].i;
                if (i >= 0) {
                    atomicAdd((unsigned long long*)&vacc[i], (unsigned long long)bs_fixed(t[v].v[0]));
                    atomicAdd((unsigned long long*)&vacc[(long long)cap + i], (unsigned long long)bs_fixed(t[v].v[1]));
                    atomicAdd((unsigned long long*)&vacc[2LL * cap + i], (unsigned long long)bs_fixed(t[v].v[2]));
                }
            }
        } else if (ns == 1) {
#pragma unroll
            for (int v = 0; v < TGT; ++v) {
                const int i = t[v].i;
                if (EOM) {
                    eom_point(ea, i, i >= 0, t[v].v[0], t[v].v[1], t[v].v[2]);
                } else if (i >= 0) {
                    vel[i] = t[v].v[0];
                    vel[(long long)cap + i] = t[v].v[1];
                    vel[2LL * cap + i] = t[v].v[2];
                }
            }
        } else {
            // partial sums by sorted position, summed in split order by the
            // last split of the target tile
#pragma unroll
            for (int v = 0; v < TGT; ++v) {
                const int k = tb * TT + threadIdx.x * TGT + v;
                if (t[v].i >= 0) {
                    part[((long long)split * 3 + 0) * cap + k] = t[v].v[0];
                    part[((long long)split * 3 + 1) * cap + k] = t[v].v[1];
                    part[((long long)split * 3 + 2) * cap + k] = t[v].v[2];
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
                    const int k = tb * TT + threadIdx.x * TGT + v, i = t[v].i;
                    float a[3] = {0.f, 0.f, 0.f};
                    if (i >= 0) {
                        for (int m = 0; m < ns; ++m)
#pragma unroll
                            for (int c = 0; c < 3; ++c) a[c] += __ldcg(&part[((long long)m * 3 + c) * cap + k]);
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

// Resident blocks: the pair loop is bound by the latency of its MUFU and
// shared-memory results and needs the warps; one target per thread fits 72
// registers (7 blocks), two 96 (5 blocks, a few spilled registers, still the
// faster form in walled boxes).
template <bool PERIODIC, int TGT, bool EOM, bool ACC>
__global__ void __launch_bounds__(BS_TPB, TGT == 1 ? 7 : 5)
    k_biot_savart(const float4* __restrict__ seg, const int* __restrict__ prev, int* __restrict__ counters,
                  int* __restrict__ tile_ticket, int cap, BoxF box, float kq, float* __restrict__ part,
                  float* __restrict__ vel, EomArgs ea, BsImages im, BsOrder o, int nsm,
                  long long* __restrict__ vacc) {
    pdl_wait_trigger();
    constexpr int NST = bs_stages<TGT>();
    __shared__ __align__(128) float4 tile[NST][BS_TILE * BS_REC];
    __shared__ __align__(8) uint64_t full[NST];
    __shared__ int release[NST], fills[NST];
    __shared__ int s_item, s_last, s_abort;
    const BsSmem sm = {NST, tile, full, release, fills, &s_item, &s_last, &s_abort};
    bs_smem_init(sm);
    uint32_t q = 0;
    const bool ok = bs_work<PERIODIC, TGT, EOM, ACC>(seg, prev, counters, tile_ticket, cap, box, kq, part, vel, ea,
                                                    im, o, nsm, sm, q, vacc);
    if (!ok && threadIdx.x == 0) {
        // a wait gave up: let every copy still in flight land before the
        // block's shared memory goes away (bounded as well)
        for (int b = 0; b < NST; ++b)
            if (fills[b] > 0) mbar_wait_bounded(&full[b], (uint32_t)(fills[b] - 1) & 1u);
    }
}

// Stand-alone entry: a caller's successor index outside [-1, n) means no
// segment (and sets the TOPOLOGY status).
__device__ __forceinline__ int bs_checked_next(const int* __restrict__ next, int n, int i) {
    const int q = next[i];
    return (q < -1 || q >= n) ? -1 : q;
}

// Stand-alone entry: prev[] of a caller's point set.
__global__ void k_bs_prev(const int* __restrict__ next, int n, int* __restrict__ prev, int* __restrict__ counters) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int q = bs_checked_next(next, n, i);
    if (q != next[i]) atomicOr(&counters[CNT_STATUS], ST_TOPOLOGY);
    if (q >= 0) prev[q] = i;
}

// Stand-alone entry: the source slots and target records of a caller's
// point set (positions [3][n]), one block per group of slots as in the
// stage geometry.
__global__ void __launch_bounds__(BS_GROUP) k_bs_points(Grid g, const double* __restrict__ pos,
                                                        const int* __restrict__ next, const int* __restrict__ prev,
                                                        int n, const int* __restrict__ counters,
                                                        float4* __restrict__ seg, BsOrder o) {
    __shared__ BsGroupSmem sm;
    const int ns = counters[CNT_NSLOT];
    const long long Np = bs_block(ns);
    const int ng = (int)(Np / BS_GROUP);
    for (int grp = blockIdx.x; grp < ng; grp += gridDim.x) {
        const int sl = grp * BS_GROUP + threadIdx.x;
        const int code = sl < ns ? o.pt[sl] : -1;
        int4 og = o.org[grp];
        const double O[3] = {(double)og.x, (double)og.y, (double)og.z};
        double rel[3] = {0.0, 0.0, 0.0};
        float d[3] = {0.f, 0.f, 0.f};
        bool jump = false;
        if (code >= 0) {
            const int q = bs_checked_next(next, n, code);
            for (int a = 0; a < 3; ++a) {
                const double si = pos[(long long)a * n + code];
                rel[a] = min_image(g, a, si - O[a]);
                if (q >= 0) {
                    const double sq = pos[(long long)a * n + q];
                    const double b = min_image(g, a, sq - si);
                    d[a] = __double2float_rn(b);
                    if (threadIdx.x != BS_GROUP - 1) jump |= fabs(min_image(g, a, sq - O[a]) - (rel[a] + b)) > 0.5;
                }
            }
        } else if (code <= -2) {
            const int q = bs_checked_next(next, n, -2 - code);
            for (int a = 0; a < 3; ++a) rel[a] = min_image(g, a, pos[(long long)a * n + q] - O[a]);
        }
        og = bs_center_origin(rel, og, sm);
        if (threadIdx.x == 0) o.org[grp] = og;
        if (code >= 0)
            bs_write_target(o.tgt, o.sorted ? o.rank[code] : code, rel, og, sl, bs_prev_slot(o, prev[code]), -1,
                            code);
        bs_write_group(0, nullptr, Np, grp, rel, d, jump, seg, sm);
    }
}

__global__ void k_bs_counters(int* __restrict__ counters, int n) {
    counters[CNT_N] = n;
    counters[CNT_STATUS] = 0;
    counters[CNT_BSWORK] = 0;
}

__global__ void k_bs_unfix(const long long* __restrict__ vacc, int n, float* __restrict__ vel) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    vel[i] = bs_value(vacc[i]);
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

int sm_count() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 152;
    }
    if (!cached[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 152;
        }
        cached[dev] = v;
    }
    return cached[dev];
}

// Up to BS_ACC_MAX points the split sums go to the fixed-point accumulator,
// so no block waits for a ticket and no last block re-reads partial sums.
bool bs_uses_vacc(int n_hint) { return n_hint < BS_ACC_MAX; }

int bs_max_splits(int cap, int nsm) {
    // the most splits: one target tile per item and every point needing a
    // gap slot (the group count only caps the splits)
    int m = 1;
    for (int n = 1; n <= cap; n += (n < 8192 ? 1 : 128)) {
        const int k = bs_splits(n, BS_TPB, nsm, (int)(bs_slot_cap(n) / BS_GROUP) * 7);
        if (k > m) m = k;
    }
    return m;
}

// Resident blocks per SM of one instantiation (queried once).
template <typename K>
int bs_resident(K kernel) {
    static int cached = 0;
    if (!cached) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, BS_TPB, 0) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 1;
        }
        cached = v;
    }
    return cached;
}

template <int TGT, bool EOM, bool ACC = false>
void bs_launch(const Grid& g, float kq, const float4* seg, const int* prev, int* cnt, int* tile_ticket, int cap, int n,
               float* part, float* vel, const EomArgs& ea, const BsImages& im, const BsOrder& o, cudaStream_t s,
               long long* vacc = nullptr) {
    // enough blocks for every item of about n points (at most the resident
    // blocks); more points than that are still covered by the blocks' item loop
    constexpr int TT = BS_TPB * TGT;
    const int nsm = sm_count();
    // at most this many items: every point with a gap slot
    const int items = ((n + TT - 1) / TT) * bs_splits(n, TT, nsm, (int)(bs_slot_cap(n) / BS_GROUP) * (1 + im.nfaces));
    const BoxF box = make_box(g);
    const bool periodic = !(g.wall[0] && g.wall[1] && g.wall[2]);
    auto kern = periodic ? k_biot_savart<true, TGT, EOM, ACC> : k_biot_savart<false, TGT, EOM, ACC>;
    const int slots = bs_resident(kern) * nsm;
    const int grid = items < slots ? items : slots;
    launch_pdl(kern, grid, BS_TPB, 0, s, seg, prev, cnt, tile_ticket, cap, box, kq, part, vel, ea, im, o, nsm, vacc);
}

void launch_biot_savart(const Grid& g, double kappa, const float4* seg, const int* prev, const int* counters,
                        int* tile_ticket, int cap, int n_hint, float* part, float* vel, cudaStream_t s,
                        const BsOrder& o, const EomArgs* eom, int nfaces, const int* face_code, const float4* geo,
                        long long* vacc) {
    if (cap <= 0) return;
    const int n = n_hint > 0 ? (n_hint < cap ? n_hint : cap) : 1;
    const float kq = (float)(kappa / (4.0 * 3.14159265358979323846));
    int* cnt = const_cast<int*>(counters);
    const EomArgs none = {};
    const EomArgs& ea = eom ? *eom : none;
    BsImages im = {};
    im.nfaces = geo ? nfaces : 0;
    const int nn[3] = {g.nx, g.ny, g.nz};
    for (int f = 0; f < im.nfaces; ++f) {
        im.face_code[f] = face_code[f];
        const int ax = face_code[f] >> 1;
        im.w2[f] = (face_code[f] & 1) ? 2.f * (float)nn[ax] - 1.f : -1.f;
    }
    // Targets per thread: from 8192 points in a box with walls on every axis,
    // 2 when the kernel applies the equation of motion (5.90 against 6.19 ms
    // per launch at 86k points in the 128x128x1024 channel: a warp has more
    // independent pairs in flight); otherwise 1
    const bool two = eom && n >= 8192 && g.wall[0] && g.wall[1] && g.wall[2];
    // without a partial-sum buffer the split sums always go to vacc
    if (vacc && !eom && (bs_uses_vacc(n) || !part)) {
        bs_launch<1, false, true>(g, kq, seg, prev, cnt, tile_ticket, cap, n, part, vel, ea, im, o, s, vacc);
        return;
    }
    if (two) bs_launch<2, true>(g, kq, seg, prev, cnt, tile_ticket, cap, n, part, vel, ea, im, o, s);
    else if (eom) bs_launch<1, true>(g, kq, seg, prev, cnt, tile_ticket, cap, n, part, vel, ea, im, o, s);
    else bs_launch<1, false>(g, kq, seg, prev, cnt, tile_ticket, cap, n, part, vel, ea, im, o, s);
}

void launch_bs_standalone_prep(const Grid& g, const double* pos, const int* next, int n, int* prev, float4* seg,
                               int* counters, const BsOrder& o, int* key, int* hist, int* bsum, cudaStream_t s) {
    k_bs_counters<<<1, 1, 0, s>>>(counters, n);
    cudaMemsetAsync(prev, 0xff, sizeof(int) * (size_t)n, s);  // first points of open lines keep -1
    k_bs_prev<<<(n + 255) / 256, 256, 0, s>>>(next, n, prev, counters);
    // the caller's positions are SoA [3][n]
    if (o.sorted)
        launch_bs_sort(g, pos, n, counters, key, hist, const_cast<int*>(o.ord), const_cast<int*>(o.rank), s);
    launch_bs_slots(pos, next, n, n, counters, o, bsum, s);
    k_bs_points<<<(int)(bs_slot_cap(n) / BS_GROUP), BS_GROUP, 0, s>>>(g, pos, next, prev, n, counters, seg, o);
}

void launch_bs_unfix(const long long* vacc, int n, float* vel, cudaStream_t s) {
    if (n > 0) k_bs_unfix<<<(3 * n + 255) / 256, 256, 0, s>>>(vacc, n, vel);
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
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(19) << 20;
// the scratch of the stand-alone entry grows linearly with the point count,
// so the array holds every call up to the point limit
static_assert(vlb::bs_scratch_bytes(NOALLOC_MAX_POINTS) <= NOALLOC_SCRATCH_BYTES,
              "the allocation-free scratch array is smaller than the scratch of its largest call");
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
