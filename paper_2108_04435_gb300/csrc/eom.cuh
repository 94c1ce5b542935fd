// Equation of motion of one filament point at one RK4 stage (Sec. II.A,
// Eqs. 4, 10-11), shared by the stand-alone kernel in vfm.cu and the
// Biot-Savart kernel in bs.cu, which applies it to each target tile as soon as
// the tile's sum is complete.
#pragma once

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

__device__ __forceinline__ void wrap_or_clamp(const Grid& g, double dmin, double s[3]) {
    for (int a = 0; a < 3; ++a) {
        const double L = (double)(a == 0 ? g.nx : (a == 1 ? g.ny : g.nz));
        if (!g.wall[a]) {
            if (s[a] < 0.0) s[a] += L;
            else if (s[a] >= L) s[a] -= L;
        } else {
            const double lo = -0.5 + 0.5 * dmin, hi = L - 0.5 - 0.5 * dmin;
            if (s[a] < lo) s[a] = lo;
            if (s[a] > hi) s[a] = hi;
        }
    }
}

// The first wall clamp bound that position s touches, in the order x-, x+,
// y-, y+, z-, z+, as 2*axis + side (side 1 = high wall), or -1.  An open end
// of a line is pinned to this wall.
__device__ __forceinline__ int touching_wall(const Grid& g, double dmin, const double s[3]) {
    for (int a = 0; a < 3; ++a) {
        if (!g.wall[a]) continue;
        const double L = (double)(a == 0 ? g.nx : (a == 1 ? g.ny : g.nz));
        if (s[a] <= -0.5 + 0.5 * dmin) return 2 * a;
        if (s[a] >= L - 0.5 - 0.5 * dmin) return 2 * a + 1;
    }
    return -1;
}

// Nodes and weights of the 2-point delta function (Eq. 11) along one axis:
// periodic axes wrap, wall axes move an outside node's weight to the nearest
// fluid node.  b = floor(s) before wrapping or clamping: points with equal b
// on every axis have the same eight nodes.
__device__ __forceinline__ void delta_axis(const Grid& g, int axis, double s, int& i0, int& i1, double& w0,
                                           double& w1, int& b) {
    const int n = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
    const double fl = floor(s);
    b = (int)fl;
    const double fr = s - fl;
    w0 = 1.0 - fr;
    w1 = fr;
    int a0 = b, a1 = b + 1;
    if (!g.wall[axis]) {
        a0 = ((a0 % n) + n) % n;
        a1 = ((a1 % n) + n) % n;
    } else {
        a0 = a0 < 0 ? 0 : (a0 > n - 1 ? n - 1 : a0);
        a1 = a1 < 0 ? 0 : (a1 > n - 1 ? n - 1 : a1);
    }
    i0 = a0;
    i1 = a1;
}

// Equation of motion (Eq. 4) at one RK4 stage, in FP32, with the
// Biot-Savart partial sums reduced in a fixed order, the local term, V_s of
// Eq. 18 as the applied superfluid flow and v_n interpolated with Eq. 11; the
// RK4 combination and the positions stay FP64.  Stage 0 also spreads the
// reaction of Eq. 10 (when spread != 0) with warp-aggregated atomics, so all
// 32 lanes of a warp must call it together (valid = false on idle lanes).
// vb = the point's Biot-Savart velocity.
__device__ __forceinline__ void eom_point(const EomArgs& A, int i, bool valid, float vbx, float vby, float vbz) {
    const VfmParams& P = A.P;
    const int stage = A.stage, spread = A.spread, cap = A.cap;
    const double* __restrict__ s0 = A.s0;
    double* __restrict__ st = A.st;
    double* __restrict__ acc = A.acc;
    const float4* __restrict__ geo = A.geo;
    const float* __restrict__ U = A.U;
    const double* __restrict__ Vs = A.Vs;
    long long* __restrict__ F = A.F;
    const Grid& g = P.g;
    const long long C = g.ncell;
    const double* xs = stage == 0 ? s0 : st;
    float s1[3] = {0.f, 0.f, 0.f}, fr[3] = {0.f, 0.f, 0.f}, dxi = 0.f;
    int ix[2] = {0, 0}, iy[2] = {0, 0}, iz[2] = {0, 0}, base[3] = {0, 0, 0};
    float wx[2] = {0.f, 0.f}, wy[2] = {0.f, 0.f}, wz[2] = {0.f, 0.f};
    if (valid) {
        double x[3];
        float vs[3];
        const float4 g0 = geo[2LL * i], g1 = geo[2LL * i + 1];
        s1[0] = g0.x; s1[1] = g0.y; s1[2] = g0.z; dxi = g0.w;
        const int pin = (int)g1.w - 1;  // wall code of a pinned end, else -1
        const float lia[3] = {g1.x, g1.y, g1.z};
        for (int k = 0; k < 3; ++k) {
            x[k] = xs[(long long)k * cap + i];
            vs[k] = (k == 0 ? vbx : (k == 1 ? vby : vbz)) + lia[k];
        }
        double w0, w1;
        delta_axis(g, 0, x[0], ix[0], ix[1], w0, w1, base[0]); wx[0] = (float)w0; wx[1] = (float)w1;
        delta_axis(g, 1, x[1], iy[0], iy[1], w0, w1, base[1]); wy[0] = (float)w0; wy[1] = (float)w1;
        delta_axis(g, 2, x[2], iz[0], iz[1], w0, w1, base[2]); wz[0] = (float)w0; wz[1] = (float)w1;
        vs[2] += wz[0] * (float)Vs[iz[0]] + wz[1] * (float)Vs[iz[1]];  // v_s,a (Eq. 18)
        float vn[3] = {0.f, 0.f, 0.f};
        for (int cz = 0; cz < 2; ++cz)
            for (int cy = 0; cy < 2; ++cy)
                for (int cx = 0; cx < 2; ++cx) {
                    const float w = wz[cz] * wy[cy] * wx[cx];
                    const long long c = ((long long)iz[cz] * g.ny + iy[cy]) * g.nx + ix[cx];
                    vn[0] += w * U[c];
                    vn[1] += w * U[C + c];
                    vn[2] += w * U[2 * C + c];
                }
        const float w[3] = {vn[0] - vs[0], vn[1] - vs[1], vn[2] - vs[2]};
        const float t[3] = {s1[1] * w[2] - s1[2] * w[1], s1[2] * w[0] - s1[0] * w[2], s1[0] * w[1] - s1[1] * w[0]};
        const float tt[3] = {s1[1] * t[2] - s1[2] * t[1], s1[2] * t[0] - s1[0] * t[2], s1[0] * t[1] - s1[1] * t[0]};
        double kv[3];
        int bad = 0;
        for (int k = 0; k < 3; ++k) {
            fr[k] = P.alpha_f * t[k] - P.alpha_p_f * tt[k];
            kv[k] = (double)(vs[k] + fr[k]);
        }
        if (pin >= 0) {  // a pinned end slides along its wall
            const int ax = pin >> 1;
            kv[0] = ax == 0 ? 0.0 : kv[0];
            kv[1] = ax == 1 ? 0.0 : kv[1];
            kv[2] = ax == 2 ? 0.0 : kv[2];
        }
        for (int k = 0; k < 3; ++k)
            if (!(fabs(P.dt * kv[k]) < 1.0)) bad |= (kv[k] == kv[k]) ? ST_CFL : ST_NAN;
        if (bad) atomicOr(&A.counters[CNT_STATUS], bad);
        const double cst_next = stage == 0 ? 0.5 : (stage == 1 ? 0.5 : 1.0);
        const double wst = (stage == 0 || stage == 3) ? 1.0 : 2.0;
        double a3[3];
        for (int k = 0; k < 3; ++k) {
            const long long o = (long long)k * cap + i;
            a3[k] = stage == 0 ? kv[k] : acc[o] + wst * kv[k];
            acc[o] = a3[k];
            if (stage == 0 && A.first) A.vel1[o] = kv[k];
        }
        if (stage < 3) {
            for (int k = 0; k < 3; ++k) {
                const long long o = (long long)k * cap + i;
                st[o] = s0[o] + cst_next * P.dt * kv[k];
            }
        } else {
            double nsx[3];
            for (int k = 0; k < 3; ++k) nsx[k] = s0[(long long)k * cap + i] + (P.dt / 6.0) * a3[k];
            wrap_or_clamp(g, P.dmin, nsx);
            for (int k = 0; k < 3; ++k) A.pos_out[(long long)k * cap + i] = nsx[k];
        }
    }
    if (stage != 0 || !spread) return;  // uniform across the grid

    // Reaction of Eq. 10 on the normal fluid: -(rho_s/rho_n) rho0 kappa * f * dxi,
    // f = friction velocity (form 0) or friction velocity x s' (form 1).
    float gv[3] = {fr[0], fr[1], fr[2]};
    if (P.force_form == 1) {
        gv[0] = fr[1] * s1[2] - fr[2] * s1[1];
        gv[1] = fr[2] * s1[0] - fr[0] * s1[2];
        gv[2] = fr[0] * s1[1] - fr[1] * s1[0];
    }
    const float scale = valid ? P.gscale_f * dxi : 0.f;
    float val[24];
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                const float w = wz[cz] * wy[cy] * wx[cx] * scale;
                const int k = (cz * 2 + cy) * 2 + cx;
                val[3 * k] = w * gv[0];
                val[3 * k + 1] = w * gv[1];
                val[3 * k + 2] = w * gv[2];
            }
    // Lanes whose points share the unclamped base cell share all eight corners
    // (a clamped base cell would not: next to a wall, floor -1 and floor 0 both
    // clamp to node 0): sum their contributions in the lowest such lane, which
    // alone issues the atomics.
    const int lane = threadIdx.x & 31;
    const long long key = valid ? ((long long)(base[2] + 1) * (g.ny + 2) + (base[1] + 1)) * (g.nx + 2) + (base[0] + 1)
                                : -1 - (long long)lane;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    const int steps = __reduce_max_sync(0xffffffffu, (unsigned)__popc(peers)) - 1;
    unsigned rest = peers & ~(1u << leader);
    for (int r = 0; r < steps; ++r) {
        const int src = rest ? __ffs(rest) - 1 : lane;
        rest &= rest - 1;
#pragma unroll
        for (int k = 0; k < 24; ++k) {
            const float v = __shfl_sync(0xffffffffu, val[k], src);
            if (lane == leader && src != lane) val[k] += v;
        }
    }
    if (!valid || lane != leader) return;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                const int k = (cz * 2 + cy) * 2 + cx;
                const long long c = ((long long)iz[cz] * g.ny + iy[cy]) * g.nx + ix[cx];
                // fixed point: exact, order-independent sums
                atomicAdd((unsigned long long*)&F[c], (unsigned long long)force_fixed(val[3 * k]));
                atomicAdd((unsigned long long*)&F[C + c], (unsigned long long)force_fixed(val[3 * k + 1]));
                atomicAdd((unsigned long long*)&F[2 * C + c], (unsigned long long)force_fixed(val[3 * k + 2]));
                A.fmask[((iz[cz] >> TILE_SHIFT) * g.tny + (iy[cy] >> TILE_SHIFT)) * g.tnx + (ix[cx] >> TILE_SHIFT)] = 1;
            }
}

}  // namespace

}  // namespace vlb
