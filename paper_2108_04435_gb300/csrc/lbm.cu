// Lattice-Boltzmann part of the coupled step (Sec. II.B of arXiv 2108.04435):
// D3Q19 BGK pull stream-collide with the split forcing of Eq. 14a-d, halfway
// bounce-back walls, moving-wall heater links (Sec. IV), the per-plane sums
// behind Eq. 18, and the activity masks that keep force/velocity traffic to
// the tiles near filaments.
//
// Populations are stored as shifted deviations g_i = f_i - w_i rho0 in FP32;
// the arithmetic below is the paper's with f_i = g_i + w_i rho0 substituted,
// which keeps the O(u) signal of each population far above FP32 rounding.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "vlb_internal.cuh"

namespace vlb {

namespace {

// Table I, 0-based, in the order documented in vlb.h.
// Each component is packed as two bits per direction (0 -> 0, 1 -> +1, 2 -> -1),
// direction i in bits 2i..2i+1, so the table folds to immediates once the
// population loops are unrolled.
__host__ __device__ constexpr int unpack_c(unsigned long long bits, int i) {
    return ((bits >> (2 * i)) & 3ull) == 1ull ? 1 : (((bits >> (2 * i)) & 3ull) == 2ull ? -1 : 0);
}
__host__ __device__ constexpr unsigned long long pack_c(const int (&c)[19], int i = 0) {
    return i == 19 ? 0ull : ((unsigned long long)(c[i] == 1 ? 1 : (c[i] == -1 ? 2 : 0)) << (2 * i)) | pack_c(c, i + 1);
}
constexpr int TCX[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
constexpr int TCY[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
constexpr int TCZ[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
constexpr unsigned long long BX = pack_c(TCX), BY = pack_c(TCY), BZ = pack_c(TCZ);
#define CX(i) unpack_c(BX, (i))
#define CY(i) unpack_c(BY, (i))
#define CZ(i) unpack_c(BZ, (i))
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr float wgt(int i) { return i == 0 ? 1.f / 3.f : (i < 7 ? 1.f / 18.f : 1.f / 36.f); }
__host__ __device__ constexpr int wclass(int i) { return i == 0 ? 0 : (i < 7 ? 1 : 2); }
// The stored deviation is g_i = f_i - s_i with s_i = fl(w_i rho0), so
// f_i = g_i + s_i exactly; the equilibrium below is shifted by s_i, not by the
// (unrepresentable) w_i rho0, via the constants dr0 and dw.

// Stored population formats: the deviation g_i = f_i - s_i in FP32, in FP16
// scaled by 2^10 (deviations of 1e-4..1e-1 stay in the normal FP16 range; the
// power-of-two scale is exact), or in BF16.  Arithmetic is FP32 in all three.
template <int S>
struct Pop;
template <>
struct Pop<STORE_F32> {
    using T = float;
    static __device__ __forceinline__ float ld(const T* p) { return __ldg(p); }
    static __device__ __forceinline__ float ld_cs(const T* p) { return __ldcs(p); }
    static __device__ __forceinline__ float raw(T v) { return v; }
    static __device__ __forceinline__ T cv(float v) { return v; }
};
template <>
struct Pop<STORE_F16> {
    using T = __half;
    static __device__ __forceinline__ float ld(const T* p) { return __half2float(__ldg(p)) * (1.f / 1024.f); }
    static __device__ __forceinline__ float ld_cs(const T* p) { return __half2float(__ldcs(p)) * (1.f / 1024.f); }
    static __device__ __forceinline__ float raw(T v) { return __half2float(v) * (1.f / 1024.f); }
    static __device__ __forceinline__ T cv(float v) { return __float2half_rn(v * 1024.f); }
};
template <>
struct Pop<STORE_BF16> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float ld(const T* p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ float ld_cs(const T* p) { return __bfloat162float(__ldcs(p)); }
    static __device__ __forceinline__ float raw(T v) { return __bfloat162float(v); }
    static __device__ __forceinline__ T cv(float v) { return __float2bfloat16_rn(v); }
};

// Population loads and stores of the stream-collide pass.  CS: evict-first
// (cache-streaming) hints on both, so that a lattice whose population buffer
// fits in L2 leaves the filament data there (LbmParams::stream_hint).
template <int S, bool CS>
__device__ __forceinline__ float pop_ld(const typename Pop<S>::T* p) {
    return CS ? Pop<S>::ld_cs(p) : Pop<S>::ld(p);
}
template <int S, bool CS>
__device__ __forceinline__ void pop_st(typename Pop<S>::T* p, float v) {
    if (CS) __stcs(p, Pop<S>::cv(v));
    else *p = Pop<S>::cv(v);
}

__device__ __forceinline__ int tile_of(const Grid& g, int x, int y, int z) {
    return ((z >> TILE_SHIFT) * g.tny + (y >> TILE_SHIFT)) * g.tnx + (x >> TILE_SHIFT);
}

// Pull the 19 shifted populations arriving at (x, y, z) (Eq. 14d in pull
// form).  A link whose source lies beyond a wall is bounced back half-way; on
// the z faces the moving-wall term 2 w_i rho0 (c_i . u_w)/c_s^2 with
// u_w = heater e_z injects (low face) or removes (high face) normal fluid.
template <bool WX, bool WY, bool WZ, int S>
__device__ __forceinline__ void pull(const typename Pop<S>::T* __restrict__ f, const LbmParams& P, int x, int y,
                                     int z, long long cell, float g[19]) {
    const int nx = P.g.nx, ny = P.g.ny, nz = P.g.nz;
    const long long C = P.g.ncell;
    int xm = x - 1, xp = x + 1, ym = y - 1, yp = y + 1, zm = z - 1, zp = z + 1;
    bool oxm = false, oxp = false, oym = false, oyp = false, ozm = false, ozp = false;
    if (xm < 0) { if (WX) oxm = true; else xm += nx; }
    if (xp >= nx) { if (WX) oxp = true; else xp -= nx; }
    if (ym < 0) { if (WY) oym = true; else ym += ny; }
    if (yp >= ny) { if (WY) oyp = true; else yp -= ny; }
    if (zm < 0) { if (WZ) ozm = true; else zm += nz; }
    if (zp >= nz) { if (WZ) ozp = true; else zp -= nz; }
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int sx = CX(i) == 1 ? xm : (CX(i) == -1 ? xp : x);
        const int sy = CY(i) == 1 ? ym : (CY(i) == -1 ? yp : y);
        const int sz = CZ(i) == 1 ? zm : (CZ(i) == -1 ? zp : z);
        const bool ox = CX(i) == 1 ? oxm : (CX(i) == -1 ? oxp : false);
        const bool oy = CY(i) == 1 ? oym : (CY(i) == -1 ? oyp : false);
        const bool oz = CZ(i) == 1 ? ozm : (CZ(i) == -1 ? ozp : false);
        if (!(ox || oy || oz)) {
            g[i] = Pop<S>::ld(&f[(long long)i * C + ((long long)sz * ny + sy) * nx + sx]);
        } else {
            float v = Pop<S>::ld(&f[(long long)opp(i) * C + cell]);
            if (oz) v += 6.f * wgt(i) * P.rho0 * (float)CZ(i) * P.heater;
            g[i] = v;
        }
    }
}

template <int OP>
__device__ __forceinline__ float warp_reduce(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float w = __shfl_xor_sync(0xffffffffu, v, o);
        v = OP == 0 ? v + w : fmaxf(v, w);
    }
    return v;
}

// The stream-collide pass's sums for Eq. 18 and the mass and Mach checks,
// one triple per warp of the launch: the warp's sum of rho - rho0 and of u_z
// over its 32 (or 32 VEC) cells and its largest |u|^2, at
// part[((z * gridDim.x + blockIdx.x) * warps per block + warp) * 3].  The
// pass itself does no FP64 arithmetic (GB300 runs FP64 at a small fraction
// of the FP32 rate, and the pass is issue-bound with 16-bit storage); the
// plane reduction adds these partials up in FP64.
__device__ __forceinline__ void warp_partials(float s_drho, float s_uz, float s_u2, float* __restrict__ part, int z) {
    s_drho = warp_reduce<0>(s_drho);
    s_uz = warp_reduce<0>(s_uz);
    s_u2 = warp_reduce<1>(s_u2);
    if ((threadIdx.x & 31) == 0) {
        const long long w = ((long long)z * gridDim.x + blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
        float* o = part + w * 3;
        o[0] = s_drho;
        o[1] = s_uz;
        o[2] = s_u2;
    }
}

// Source index of the population arriving along c_i (pull form of
// Eq. 14d): 32-bit, from per-thread row/plane offsets (the host limits the
// lattice to 19 C < 2^31).  A link leaving through a wall is replaced by the
// opposite population of the same cell (halfway bounce-back); the moving-wall
// term of the z faces is added by the caller.
struct PullIdx {
    int xo[3], yo[3], zo[3];  // offsets for c = -1, 0, +1 (index c + 1)
    bool ox[3], oy[3], oz[3]; // source outside a wall
};

template <bool WX, bool WY, bool WZ>
__device__ __forceinline__ void pull_index(const LbmParams& P, int x, int y, int z, PullIdx& q) {
    const int nx = P.g.nx, ny = P.g.ny, nz = P.g.nz, nxy = nx * ny;
    int xm = x - 1, xp = x + 1, ym = y - 1, yp = y + 1, zm = z - 1, zp = z + 1;
    // c = +1 pulls from x - 1, c = -1 from x + 1
    q.ox[0] = q.ox[1] = q.ox[2] = false;
    q.oy[0] = q.oy[1] = q.oy[2] = false;
    q.oz[0] = q.oz[1] = q.oz[2] = false;
    if (xm < 0) { if (WX) q.ox[2] = true; else xm += nx; }
    if (xp >= nx) { if (WX) q.ox[0] = true; else xp -= nx; }
    if (ym < 0) { if (WY) q.oy[2] = true; else ym += ny; }
    if (yp >= ny) { if (WY) q.oy[0] = true; else yp -= ny; }
    if (zm < 0) { if (WZ) q.oz[2] = true; else zm += nz; }
    if (zp >= nz) { if (WZ) q.oz[0] = true; else zp -= nz; }
    q.xo[0] = xp; q.xo[1] = x; q.xo[2] = xm;
    q.yo[0] = yp * nx; q.yo[1] = y * nx; q.yo[2] = ym * nx;
    q.zo[0] = zp * nxy; q.zo[1] = z * nxy; q.zo[2] = zm * nxy;
}

template <bool WX, bool WY, bool WZ, int S, bool CS>
__device__ __forceinline__ void pull_fast(const typename Pop<S>::T* __restrict__ f, const LbmParams& P,
                                          const PullIdx& q, int cell, float g[19]) {
    const int C = (int)P.g.ncell;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        int src = i * C + q.zo[CZ(i) + 1] + q.yo[CY(i) + 1] + q.xo[CX(i) + 1];
        bool out = false, outz = false;
        if (WX && CX(i) != 0) out = out || q.ox[CX(i) + 1];
        if (WY && CY(i) != 0) out = out || q.oy[CY(i) + 1];
        if (WZ && CZ(i) != 0) { outz = q.oz[CZ(i) + 1]; out = out || outz; }
        if (WX || WY || WZ) src = out ? opp(i) * C + cell : src;
        float v = pop_ld<S, CS>(&f[src]);
        if (WZ && CZ(i) != 0) v += outz ? 6.f * wgt(i) * P.rho0 * (float)CZ(i) * P.heater : 0.f;
        g[i] = v;
    }
}

// K1: one lattice pass.  One thread per cell, one block per 256 consecutive
// (x, y) cells of one z plane, so every population array is read in coalesced
// rows (the +-x shift of the pull is absorbed by L1/L2) and written aligned.
// The collision works on opposite pairs (i, i'): with c_i' = -c_i the even
// parts of f^eq (Eq. 7) and of F_i (Eq. 13) are shared and the odd parts
// change sign.
template <bool WX, bool WY, bool WZ, int S, bool CS>
__global__ void __launch_bounds__(LBM_BLOCK) k_lbm_step(const typename Pop<S>::T* __restrict__ fin,
                                                        typename Pop<S>::T* __restrict__ fout,
                                                        const long long* __restrict__ F, float* __restrict__ U,
                                                        const uint8_t* __restrict__ fmask,
                                                        const uint8_t* __restrict__ umask, float* __restrict__ part,
                                                        LbmParams P) {
    pdl_wait_trigger();
    const int nx = P.g.nx, ny = P.g.ny;
    const int C = (int)P.g.ncell;
    const int z = blockIdx.y;
    const int xy = blockIdx.x * blockDim.x + threadIdx.x;
    float s_drho = 0.f, s_uz = 0.f, s_u2 = 0.f;
    if (xy < nx * ny) {
        const int y = (int)(((unsigned long long)(unsigned)xy * P.nx_magic) >> P.nx_shift), x = xy - y * nx;
        const int cell = z * nx * ny + xy;
        float g[19];
        {
            PullIdx q;
            pull_index<WX, WY, WZ>(P, x, y, z, q);
            pull_fast<WX, WY, WZ, S, CS>(fin, P, q, cell, g);
        }
        // Eqs. 5-6 with the half-force shift: rho = rho0 + sum g, j = sum c g
        float drho = P.dr0, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            drho += g[i];
            if (CX(i)) jx += (float)CX(i) * g[i];
            if (CY(i)) jy += (float)CY(i) * g[i];
            if (CZ(i)) jz += (float)CZ(i) * g[i];
        }
        const int tile = tile_of(P.g, x, y, z);
        const bool factive = fmask[tile] != 0;
        float Fx = P.body[0], Fy = P.body[1], Fz = P.body[2];
        if (factive) {
            Fx += force_value(__ldg(&F[cell]));
            Fy += force_value(__ldg(&F[C + cell]));
            Fz += force_value(__ldg(&F[2 * C + cell]));
        }
        const bool force = factive || P.body_on;
        const float rho = P.rho0 + drho;
        const float inv = __fdividef(1.f, rho);  // ~1 ulp; rho is close to rho0
        const float ux = (jx + 0.5f * Fx) * inv, uy = (jy + 0.5f * Fy) * inv, uz = (jz + 0.5f * Fz) * inv;
        const float usq = ux * ux + uy * uy + uz * uz;
        if (P.all_u || umask[tile]) {
            U[cell] = ux;
            U[C + cell] = uy;
            U[2 * C + cell] = uz;
        }
        const float om = P.omega;
        const float A = drho - 1.5f * rho * usq;  // even part of f^eq/w - rho0 without the (c.u)^2 term
        const float B3 = 3.f * rho, B45 = 4.5f * rho;
        const float uF = ux * Fx + uy * Fy + uz * Fz;
        const bool pinned = P.pin_on && z == 0;
        // rest population
        {
            float geq = wgt(0) * A + P.dw[0];
            float out = g[0] + om * (geq - g[0]);
            if (force) out += P.pref * wgt(0) * (-3.f * uF);
            if (pinned) out = wgt(0) * (drho - 1.5f * rho * P.pin * P.pin) + P.dw[0];
            pop_st<S, CS>(&fout[cell], out);
        }
#pragma unroll
        for (int i = 1; i < 19; i += 2) {
            const int j = i + 1;  // opposite of i
            const float cu = (float)CX(i) * ux + (float)CY(i) * uy + (float)CZ(i) * uz;
            const float w = wgt(i);
            const float sym = w * (A + B45 * cu * cu) + P.dw[wclass(i)];
            const float asym = w * B3 * cu;
            float oi = g[i] + om * (sym + asym - g[i]);
            float oj = g[j] + om * (sym - asym - g[j]);
            if (force) {
                const float cF = (float)CX(i) * Fx + (float)CY(i) * Fy + (float)CZ(i) * Fz;
                const float fs = P.pref * w * (9.f * cu * cF - 3.f * uF);
                const float fa = P.pref * w * 3.f * cF;
                oi += fs + fa;
                oj += fs - fa;
            }
            if (pinned) {
                const float cp = (float)CZ(i) * P.pin;
                const float ps = w * (drho + rho * (4.5f * cp * cp - 1.5f * P.pin * P.pin)) + P.dw[wclass(i)];
                const float pa = w * B3 * cp;
                oi = ps + pa;
                oj = ps - pa;
            }
            pop_st<S, CS>(&fout[i * C + cell], oi);
            pop_st<S, CS>(&fout[j * C + cell], oj);
        }
        s_drho = drho;
        s_uz = uz;
        s_u2 = (usq == usq) ? usq : INFINITY;
    }
    // per-warp partials for Eq. 18 and the mass / Mach checks (summed in
    // FP64 by the plane reduction)
    warp_partials(s_drho, s_uz, s_u2, part, z);
}

// Eq. 18 per z plane from the stream-collide warp partials (FP32, added up
// here in FP64), with the mass and the Mach limit of Sec. II.B
// (|u|/c_s < 0.05).  One warp per plane (lane-strided loads, fixed shuffle
// tree); the last block to finish reduces
// the planes in a fixed order.  FP64 work is spread over many SMs because
// its per-SM rate is low on this GPU.  The stream-collide pass has consumed
// the force grid: one warp per tile resets it in the flagged tiles, then
// both tile flags are cleared for the next step.  The first nplane blocks
// hold the plane warps; the grid has enough blocks beyond them for about
// one tile per warp, since a warp that resets tile after tile is a long
// chain of dependent address arithmetic and stores.
__global__ void __launch_bounds__(256) k_plane_vs(const float* __restrict__ part, int wpp, LbmParams P,
                                                  long long* __restrict__ F, uint8_t* __restrict__ umask,
                                                  uint8_t* __restrict__ fmask, int ntiles, int nplane) {
    pdl_wait_trigger();
    {
        const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nwarps = (int)((gridDim.x * blockDim.x) >> 5);
        const int ln = threadIdx.x & 31;
        const Grid& g = P.g;
        for (int t = warp; t < ntiles; t += nwarps) {
            if (fmask[t]) {
                const int tx = t % g.tnx, ty = (t / g.tnx) % g.tny, tz = t / (g.tnx * g.tny);
#pragma unroll 4
                for (int k = ln; k < 512; k += 32) {
                    const int x = (tx << TILE_SHIFT) + (k & 7), y = (ty << TILE_SHIFT) + ((k >> 3) & 7),
                              z = (tz << TILE_SHIFT) + (k >> 6);
                    if (x < g.nx && y < g.ny && z < g.nz) {
                        const long long c = ((long long)z * g.ny + y) * g.nx + x;
                        F[c] = 0;
                        F[g.ncell + c] = 0;
                        F[2 * g.ncell + c] = 0;
                    }
                }
                __syncwarp();
                if (ln == 0) fmask[t] = 0;
            }
            if (ln == 0) umask[t] = 0;
        }
    }
    if ((int)blockIdx.x >= nplane) return;  // a tile-only block (uniform)
    __shared__ double s_tot[256], s_mass[256], s_max[256];
    __shared__ int s_last;
    const int nz = P.g.nz;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int pz = blockIdx.x * 8 + wid;
    if (pz < nz) {
        double a = 0.0, b = 0.0, m = 0.0;
        for (int k = lane; k < wpp; k += 32) {
            const float* o = part + ((long long)pz * wpp + k) * 3;
            a += (double)o[0];
            b += (double)o[1];
            m = fmax(m, (double)o[2]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, off);
            b += __shfl_xor_sync(0xffffffffu, b, off);
            m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
        }
        if (lane == 0) {
            double* pl = P.plane + 3LL * pz;
            pl[0] = a;
            pl[1] = b;
            pl[2] = m;
            if (P.g.wall[2]) P.Vs[pz] = -P.inv_ratio * (b / ((double)P.g.nx * (double)P.g.ny));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&P.counters[CNT_PLANES], 1) == nplane - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double tot = 0.0, mass = 0.0, mx = 0.0;
    for (int q = threadIdx.x; q < nz; q += blockDim.x) {
        const double* pl = P.plane + 3LL * q;
        mass += __ldcg(&pl[0]);
        tot += __ldcg(&pl[1]);
        mx = fmax(mx, __ldcg(&pl[2]));
    }
    s_tot[threadIdx.x] = tot;
    s_mass[threadIdx.x] = mass;
    s_max[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s_tot[threadIdx.x] += s_tot[threadIdx.x + o];
            s_mass[threadIdx.x] += s_mass[threadIdx.x + o];
            s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (!P.g.wall[2]) {
        const double v = -P.inv_ratio * (s_tot[0] / (double)P.g.ncell);
        for (int q = threadIdx.x; q < nz; q += blockDim.x) P.Vs[q] = v;
    }
    if (threadIdx.x == 0) {
        const double m = s_max[0];
        const double mach = sqrt(3.0 * m);
        P.dstats[DS_MASS] = (double)P.rho0 * (double)P.g.ncell + s_mass[0];
        P.dstats[DS_MAXMACH] = mach;
        int st = 0;
        if (!(mach < 0.05)) st |= ST_MACH;
        if (!isfinite(m) || !isfinite(s_mass[0])) st |= ST_NAN;
        if (st) atomicOr(&P.counters[CNT_STATUS], st);
        P.counters[CNT_PLANES] = 0;
    }
}

// K1, vectorised: each thread owns VEC consecutive x-cells of one row and
// loads every population row segment with one VEC-wide load.  The +-x
// shifted populations come from the neighbouring lane (the previous or next
// VEC cells of the same row) by a shuffle, with a scalar load only at warp
// and row edges; links leaving through a wall are bounced back from the
// cell's own opposite population.  Requires nx % VEC == 0.
template <int VEC>
struct VecT;
template <>
struct VecT<2> {
    using T = float2;
};
template <>
struct VecT<4> {
    using T = float4;
};

template <int VEC>
__device__ __forceinline__ void vload(const float* __restrict__ p, float (&v)[VEC]) {
    const typename VecT<VEC>::T t = __ldg(reinterpret_cast<const typename VecT<VEC>::T*>(p));
    const float* q = reinterpret_cast<const float*>(&t);
#pragma unroll
    for (int c = 0; c < VEC; ++c) v[c] = q[c];
}

template <int VEC>
__device__ __forceinline__ void vstore(float* p, const float (&v)[VEC]) {
    typename VecT<VEC>::T t;
    float* q = reinterpret_cast<float*>(&t);
#pragma unroll
    for (int c = 0; c < VEC; ++c) q[c] = v[c];
    *reinterpret_cast<typename VecT<VEC>::T*>(p) = t;
}

template <bool WX, bool WY, bool WZ, int VEC>
__global__ void __launch_bounds__(128) k_lbm_step_vec(const float* __restrict__ fin, float* __restrict__ fout,
                                                      const long long* __restrict__ F, float* __restrict__ U,
                                                      const uint8_t* __restrict__ fmask,
                                                      const uint8_t* __restrict__ umask, float* __restrict__ part,
                                                      LbmParams P) {
    pdl_wait_trigger();
    const int nx = P.g.nx, ny = P.g.ny, nz = P.g.nz, nxy = nx * ny;
    const int C = (int)P.g.ncell;
    const int nq = nx / VEC;  // cell groups per row
    const int z = blockIdx.y;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool live = q < nq * ny;
    const int y = live ? q / nq : 0;
    const int x0 = live ? (q - y * nq) * VEC : 0;
    const int cell0 = z * nxy + y * nx + x0;
    // source rows for c_y, c_z = -1, 0, +1 (index c + 1); out = beyond a wall
    int ym = y - 1, yp = y + 1, zm = z - 1, zp = z + 1;
    bool oym = false, oyp = false, ozm = false, ozp = false;
    if (ym < 0) { if (WY) oym = true; else ym += ny; }
    if (yp >= ny) { if (WY) oyp = true; else yp -= ny; }
    if (zm < 0) { if (WZ) ozm = true; else zm += nz; }
    if (zp >= nz) { if (WZ) ozp = true; else zp -= nz; }
    const int yo[3] = {yp * nx, y * nx, ym * nx};
    const int zo[3] = {zp * nxy, z * nxy, zm * nxy};
    const bool oy[3] = {oyp, false, oym};
    const bool oz[3] = {ozp, false, ozm};
    const bool row_first = x0 == 0, row_last = x0 + VEC == nx;

    // Phase 1: every load of the cell group is issued before any is used:
    // the VEC-wide row segments and, for edge lanes, the scalar value beyond
    // the segment that the neighbouring lane cannot supply.
    float g[19][VEC];
    float edge[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int row = i * C + zo[CZ(i) + 1] + yo[CY(i) + 1];
        const bool rowout = (WY && oy[CY(i) + 1]) || (WZ && oz[CZ(i) + 1]);
        if (live) {
            vload<VEC>(rowout ? fin + opp(i) * C + cell0 : fin + row + x0, g[i]);
        } else {
#pragma unroll
            for (int c = 0; c < VEC; ++c) g[i][c] = 0.f;
        }
        edge[i] = 0.f;
        if (CX(i) == 1) {
            const bool need = live && !rowout && (lane == 0 || row_first);
            const int a = !row_first ? row + x0 - 1 : (WX ? opp(i) * C + cell0 : row + nx - 1);
            if (need) edge[i] = __ldg(&fin[a]);
        } else if (CX(i) == -1) {
            const bool need = live && !rowout && (lane == 31 || row_last);
            const int a = !row_last ? row + x0 + VEC : (WX ? opp(i) * C + cell0 + VEC - 1 : row);
            if (need) edge[i] = __ldg(&fin[a]);
        }
    }
    // Phase 2: moving-wall terms, then the +-x shifts through the neighbouring lanes.
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const bool rowout = (WY && oy[CY(i) + 1]) || (WZ && oz[CZ(i) + 1]);
        if (WZ && CZ(i) != 0 && oz[CZ(i) + 1]) {
            const float h = 6.f * wgt(i) * P.rho0 * (float)CZ(i) * P.heater;
#pragma unroll
            for (int c = 0; c < VEC; ++c) g[i][c] += h;
        }
        if (CX(i) == 1) {
            // cells x0..x0+VEC-1 pull from x0-1..x0+VEC-2
            const float nb = __shfl_up_sync(0xffffffffu, g[i][VEC - 1], 1);
            const float left = (lane == 0 || row_first) ? edge[i] : nb;
            if (!rowout) {
#pragma unroll
                for (int c = VEC - 1; c > 0; --c) g[i][c] = g[i][c - 1];
                g[i][0] = left;
            }
        } else if (CX(i) == -1) {
            // cells x0..x0+VEC-1 pull from x0+1..x0+VEC
            const float nb = __shfl_down_sync(0xffffffffu, g[i][0], 1);
            const float right = (lane == 31 || row_last) ? edge[i] : nb;
            if (!rowout) {
#pragma unroll
                for (int c = 0; c < VEC - 1; ++c) g[i][c] = g[i][c + 1];
                g[i][VEC - 1] = right;
            }
        }
    }

    float s_drho = 0.f, s_uz = 0.f, s_u2 = 0.f;
    if (live) {
        const int tile = tile_of(P.g, x0, y, z);  // VEC <= 8 cells share a tile
        const bool factive = fmask[tile] != 0;
        const bool force = factive || P.body_on;
        const bool uact = P.all_u || umask[tile] != 0;
        float Fx[VEC], Fy[VEC], Fz[VEC];
#pragma unroll
        for (int c = 0; c < VEC; ++c) {
            Fx[c] = P.body[0];
            Fy[c] = P.body[1];
            Fz[c] = P.body[2];
        }
        if (factive) {
#pragma unroll
            for (int c = 0; c < VEC; ++c) {
                Fx[c] += force_value(F[cell0 + c]);
                Fy[c] += force_value(F[C + cell0 + c]);
                Fz[c] += force_value(F[2 * C + cell0 + c]);
            }
        }
        float drho[VEC], ux[VEC], uy[VEC], uz[VEC];
#pragma unroll
        for (int c = 0; c < VEC; ++c) {
            // Eqs. 5-6 with the half-force shift
            float d = P.dr0, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
            for (int i = 0; i < 19; ++i) {
                d += g[i][c];
                if (CX(i)) jx += (float)CX(i) * g[i][c];
                if (CY(i)) jy += (float)CY(i) * g[i][c];
                if (CZ(i)) jz += (float)CZ(i) * g[i][c];
            }
            const float inv = 1.f / (P.rho0 + d);
            drho[c] = d;
            ux[c] = (jx + 0.5f * Fx[c]) * inv;
            uy[c] = (jy + 0.5f * Fy[c]) * inv;
            uz[c] = (jz + 0.5f * Fz[c]) * inv;
        }
        if (uact) {
            vstore<VEC>(U + cell0, ux);
            vstore<VEC>(U + C + cell0, uy);
            vstore<VEC>(U + 2 * C + cell0, uz);
        }
        const float om = P.omega;
        const bool pinned = P.pin_on && z == 0;
        float A[VEC], B3[VEC], B45[VEC], uF[VEC];
#pragma unroll
        for (int c = 0; c < VEC; ++c) {
            const float rho = P.rho0 + drho[c];
            const float usq = ux[c] * ux[c] + uy[c] * uy[c] + uz[c] * uz[c];
            A[c] = drho[c] - 1.5f * rho * usq;
            B3[c] = 3.f * rho;
            B45[c] = 4.5f * rho;
            uF[c] = ux[c] * Fx[c] + uy[c] * Fy[c] + uz[c] * Fz[c];
            s_drho += drho[c];
            s_uz += uz[c];
            s_u2 = fmaxf(s_u2, (usq == usq) ? usq : INFINITY);
        }
        // rest population
#pragma unroll
        for (int c = 0; c < VEC; ++c) {
            float out = g[0][c] + om * (wgt(0) * A[c] + P.dw[0] - g[0][c]);
            if (force) out += P.pref * wgt(0) * (-3.f * uF[c]);
            if (pinned) out = wgt(0) * (drho[c] - 1.5f * (P.rho0 + drho[c]) * P.pin * P.pin) + P.dw[0];
            g[0][c] = out;
        }
        vstore<VEC>(fout + cell0, g[0]);
        // opposite pairs (i, i+1): even parts of Eqs. 7 and 13 shared, odd parts change sign
#pragma unroll
        for (int i = 1; i < 19; i += 2) {
            const int j = i + 1;
            const float w = wgt(i);
#pragma unroll
            for (int c = 0; c < VEC; ++c) {
                const float cu = (float)CX(i) * ux[c] + (float)CY(i) * uy[c] + (float)CZ(i) * uz[c];
                const float sym = w * (A[c] + B45[c] * cu * cu) + P.dw[wclass(i)];
                const float asym = w * B3[c] * cu;
                float oi = g[i][c] + om * (sym + asym - g[i][c]);
                float oj = g[j][c] + om * (sym - asym - g[j][c]);
                if (force) {
                    const float cF = (float)CX(i) * Fx[c] + (float)CY(i) * Fy[c] + (float)CZ(i) * Fz[c];
                    const float fs = P.pref * w * (9.f * cu * cF - 3.f * uF[c]);
                    const float fa = P.pref * w * 3.f * cF;
                    oi += fs + fa;
                    oj += fs - fa;
                }
                if (pinned) {
                    const float cp = (float)CZ(i) * P.pin;
                    const float rho = P.rho0 + drho[c];
                    const float ps =
                        w * (drho[c] + rho * (4.5f * cp * cp - 1.5f * P.pin * P.pin)) + P.dw[wclass(i)];
                    const float pa = w * B3[c] * cp;
                    oi = ps + pa;
                    oj = ps - pa;
                }
                g[i][c] = oi;
                g[j][c] = oj;
            }
            vstore<VEC>(fout + i * C + cell0, g[i]);
            vstore<VEC>(fout + j * C + cell0, g[j]);
        }
    }
    // per-warp partials for Eq. 18 and the mass / Mach checks
    warp_partials(s_drho, s_uz, s_u2, part, z);
}

// Two adjacent 16-bit populations (the first at an even x, so 4-byte
// aligned) as floats, and back: one 32-bit load or store for both cells.
template <int S>
struct Pop2;
template <>
struct Pop2<STORE_F16> {
    using T2 = __half2;
    static __device__ __forceinline__ float2 ld(const __half* p, bool cs) {
        const __half2* q = reinterpret_cast<const __half2*>(p);
        return __fmul2_rn(__half22float2(cs ? __ldcs(q) : __ldg(q)), make_float2(1.f / 1024.f, 1.f / 1024.f));
    }
    static __device__ __forceinline__ void st(__half* p, float2 v, bool cs) {
        const __half2 h = __float22half2_rn(__fmul2_rn(v, make_float2(1024.f, 1024.f)));
        __half2* q = reinterpret_cast<__half2*>(p);
        if (cs) __stcs(q, h);
        else *q = h;
    }
};
template <>
struct Pop2<STORE_BF16> {
    using T2 = __nv_bfloat162;
    static __device__ __forceinline__ float2 ld(const __nv_bfloat16* p, bool cs) {
        const __nv_bfloat162* q = reinterpret_cast<const __nv_bfloat162*>(p);
        return __bfloat1622float2(cs ? __ldcs(q) : __ldg(q));
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float2 v, bool cs) {
        const __nv_bfloat162 h = __float22bfloat162_rn(v);
        __nv_bfloat162* q = reinterpret_cast<__nv_bfloat162*>(p);
        if (cs) __stcs(q, h);
        else *q = h;
    }
};

__device__ __forceinline__ float2 f2c(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// K1 for 16-bit population storage: two adjacent cells (x even) per thread.
// With 16-bit populations the one-cell kernel is bound by instruction issue
// (a 2-byte load, two conversions and their address arithmetic per value),
// not by HBM; here each population of both cells is one aligned 32-bit load
// and one 32-bit store, a +-x shifted population adds one 2-byte load of the
// value beyond the pair (from L1: the neighbouring thread loads that line),
// and the collision runs on both cells at once in packed FP32x2 arithmetic.
// Same equations and operation order per cell as k_lbm_step.  Every load is
// issued unconditionally from an address that is valid for every thread (a
// link through a wall reads the cell's own opposite population; a thread
// past the lattice reads the plane's first cells), so all 29 loads of a
// thread are in flight together: with the loads under per-thread conditions
// the walled kernel ran at half the speed of the periodic one.  Requires an
// even nx; 128 threads (256 cells) per block.
template <bool WX, bool WY, bool WZ, int S, bool CS>
__device__ __forceinline__ void lbm_pair_cells(const typename Pop<S>::T* __restrict__ fin,
                                               typename Pop<S>::T* __restrict__ fout,
                                               const long long* __restrict__ F, float* __restrict__ U,
                                               const uint8_t* __restrict__ fmask,
                                               const uint8_t* __restrict__ umask, const LbmParams& P, int z, int q,
                                               float& s_drho, float& s_uz, float& s_u2) {
    const int nx = P.g.nx, ny = P.g.ny, nz = P.g.nz, nxy = nx * ny;
    const int C = (int)P.g.ncell;
    const int nq = nx / 2;  // cell pairs per row
    const bool live = q < nq * ny;
    const int y = live ? q / nq : 0;
    const int x0 = live ? (q - y * nq) * 2 : 0;
    const int cell0 = z * nxy + y * nx + x0;
    int ym = y - 1, yp = y + 1, zm = z - 1, zp = z + 1;
    bool oym = false, oyp = false, ozm = false, ozp = false;
    if (ym < 0) { if (WY) oym = true; else ym += ny; }
    if (yp >= ny) { if (WY) oyp = true; else yp -= ny; }
    if (zm < 0) { if (WZ) ozm = true; else zm += nz; }
    if (zp >= nz) { if (WZ) ozp = true; else zp -= nz; }
    const int yo[3] = {yp * nx, y * nx, ym * nx};
    const int zo[3] = {zp * nxy, z * nxy, zm * nxy};
    const bool oy[3] = {oyp, false, oym};
    const bool oz[3] = {ozp, false, ozm};
    const bool row_first = x0 == 0, row_last = x0 + 2 == nx;

    // every load first: the aligned pair of the source row (or, beyond a y or
    // z wall, the opposite populations of the same two cells), and for a +-x
    // shift the value beyond the pair (x0 - 1 or x0 + 2, the row's other end
    // on a periodic x axis, the cell's own opposite population at an x wall)
    float2 g[19];
    float edge[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int row = i * C + zo[CZ(i) + 1] + yo[CY(i) + 1];
        const bool rowout = (WY && oy[CY(i) + 1]) || (WZ && oz[CZ(i) + 1]);
        const int src = rowout ? opp(i) * C + cell0 : row + x0;
        g[i] = Pop2<S>::ld(fin + src, CS);
        edge[i] = 0.f;
        if (CX(i) == 1) {
            int a = !row_first ? row + x0 - 1 : (WX ? opp(i) * C + cell0 : row + nx - 1);
            a = rowout ? src : a;
            edge[i] = pop_ld<S, CS>(&fin[a]);
        } else if (CX(i) == -1) {
            int a = !row_last ? row + x0 + 2 : (WX ? opp(i) * C + cell0 + 1 : row);
            a = rowout ? src : a;
            edge[i] = pop_ld<S, CS>(&fin[a]);
        }
    }
    // moving-wall terms, then the +-x shifts
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const bool rowout = (WY && oy[CY(i) + 1]) || (WZ && oz[CZ(i) + 1]);
        if (WZ && CZ(i) != 0 && oz[CZ(i) + 1]) g[i] = add2(g[i], f2c(6.f * wgt(i) * P.rho0 * (float)CZ(i) * P.heater));
        if (CX(i) == 1) {
            // cells x0, x0 + 1 pull from x0 - 1, x0
            if (!rowout) g[i] = make_float2(edge[i], g[i].x);
        } else if (CX(i) == -1) {
            // cells x0, x0 + 1 pull from x0 + 1, x0 + 2
            if (!rowout) g[i] = make_float2(g[i].y, edge[i]);
        }
    }
    if (live) {
        const int tile = tile_of(P.g, x0, y, z);  // both cells share a tile
        const bool factive = fmask[tile] != 0;
        const bool force = factive || P.body_on;
        const bool uact = P.all_u || umask[tile] != 0;
        float2 Fx = f2c(P.body[0]), Fy = f2c(P.body[1]), Fz = f2c(P.body[2]);
        if (factive) {
            const longlong2 fx = __ldg(reinterpret_cast<const longlong2*>(F + cell0));
            const longlong2 fy = __ldg(reinterpret_cast<const longlong2*>(F + C + cell0));
            const longlong2 fz = __ldg(reinterpret_cast<const longlong2*>(F + 2 * C + cell0));
            Fx = add2(Fx, make_float2(force_value(fx.x), force_value(fx.y)));
            Fy = add2(Fy, make_float2(force_value(fy.x), force_value(fy.y)));
            Fz = add2(Fz, make_float2(force_value(fz.x), force_value(fz.y)));
        }
        // Eqs. 5-6 with the half-force shift: rho = rho0 + sum g, j = sum c g
        float2 drho = f2c(P.dr0), jx = f2c(0.f), jy = f2c(0.f), jz = f2c(0.f);
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            drho = add2(drho, g[i]);
            if (CX(i)) jx = CX(i) > 0 ? add2(jx, g[i]) : sub2(jx, g[i]);
            if (CY(i)) jy = CY(i) > 0 ? add2(jy, g[i]) : sub2(jy, g[i]);
            if (CZ(i)) jz = CZ(i) > 0 ? add2(jz, g[i]) : sub2(jz, g[i]);
        }
        const float2 rho = add2(f2c(P.rho0), drho);
        const float2 inv = make_float2(__fdividef(1.f, rho.x), __fdividef(1.f, rho.y));
        const float2 ux = mul2(fma2(f2c(0.5f), Fx, jx), inv);
        const float2 uy = mul2(fma2(f2c(0.5f), Fy, jy), inv);
        const float2 uz = mul2(fma2(f2c(0.5f), Fz, jz), inv);
        const float2 usq = fma2(uz, uz, fma2(uy, uy, mul2(ux, ux)));
        if (uact) {
            *reinterpret_cast<float2*>(U + cell0) = ux;
            *reinterpret_cast<float2*>(U + C + cell0) = uy;
            *reinterpret_cast<float2*>(U + 2 * C + cell0) = uz;
        }
        const float2 om = f2c(P.omega);
        const float2 A = fma2(mul2(f2c(-1.5f), rho), usq, drho);  // even part of f^eq/w - rho0 without (c.u)^2
        const float2 B3 = mul2(f2c(3.f), rho), B45 = mul2(f2c(4.5f), rho);
        const float2 uF = fma2(uz, Fz, fma2(uy, Fy, mul2(ux, Fx)));
        const bool pinned = P.pin_on && z == 0;
        s_drho = drho.x + drho.y;
        s_uz = uz.x + uz.y;
        s_u2 = fmaxf((usq.x == usq.x) ? usq.x : INFINITY, (usq.y == usq.y) ? usq.y : INFINITY);
        // rest population
        {
            const float2 geq = fma2(f2c(wgt(0)), A, f2c(P.dw[0]));
            float2 out = fma2(om, sub2(geq, g[0]), g[0]);
            if (force) out = fma2(f2c(P.pref * wgt(0) * -3.f), uF, out);
            if (pinned) {
                const float2 pr = fma2(mul2(f2c(-1.5f * P.pin * P.pin), rho), f2c(1.f), drho);
                out = fma2(f2c(wgt(0)), pr, f2c(P.dw[0]));
            }
            Pop2<S>::st(fout + cell0, out, CS);
        }
        // opposite pairs (i, i + 1): even parts of Eqs. 7 and 13 shared, odd parts change sign
#pragma unroll
        for (int i = 1; i < 19; i += 2) {
            const int j = i + 1;
            const float w = wgt(i);
            float2 cu = f2c(0.f);
            if (CX(i)) cu = CX(i) > 0 ? add2(cu, ux) : sub2(cu, ux);
            if (CY(i)) cu = CY(i) > 0 ? add2(cu, uy) : sub2(cu, uy);
            if (CZ(i)) cu = CZ(i) > 0 ? add2(cu, uz) : sub2(cu, uz);
            const float2 sym = fma2(f2c(w), fma2(B45, mul2(cu, cu), A), f2c(P.dw[wclass(i)]));
            const float2 asym = mul2(mul2(f2c(w), B3), cu);
            float2 oi = fma2(om, sub2(add2(sym, asym), g[i]), g[i]);
            float2 oj = fma2(om, sub2(sub2(sym, asym), g[j]), g[j]);
            if (force) {
                float2 cF = f2c(0.f);
                if (CX(i)) cF = CX(i) > 0 ? add2(cF, Fx) : sub2(cF, Fx);
                if (CY(i)) cF = CY(i) > 0 ? add2(cF, Fy) : sub2(cF, Fy);
                if (CZ(i)) cF = CZ(i) > 0 ? add2(cF, Fz) : sub2(cF, Fz);
                const float2 fs = mul2(f2c(P.pref * w), fma2(mul2(f2c(9.f), cu), cF, mul2(f2c(-3.f), uF)));
                const float2 fa = mul2(f2c(P.pref * w * 3.f), cF);
                oi = add2(oi, add2(fs, fa));
                oj = add2(oj, sub2(fs, fa));
            }
            if (pinned) {
                const float cp = (float)CZ(i) * P.pin;
                const float2 ps = fma2(f2c(w), fma2(rho, f2c(4.5f * cp * cp - 1.5f * P.pin * P.pin), drho),
                                       f2c(P.dw[wclass(i)]));
                const float2 pa = mul2(mul2(f2c(w), B3), f2c(cp));
                oi = add2(ps, pa);
                oj = sub2(ps, pa);
            }
            Pop2<S>::st(fout + i * C + cell0, oi, CS);
            Pop2<S>::st(fout + j * C + cell0, oj, CS);
        }
    }
}

// The kernel: a block whose two rows lie off the y faces, in a plane off the
// z faces (block-uniform), takes the body without the y and z wall logic
// (every link of its cells stays inside the lattice there, so the result is
// the same); the blocks along those faces take the full body.
template <bool WX, bool WY, bool WZ, int S, bool CS>
__global__ void __launch_bounds__(128, 6) k_lbm_step_pair(const typename Pop<S>::T* __restrict__ fin,
                                                       typename Pop<S>::T* __restrict__ fout,
                                                       const long long* __restrict__ F, float* __restrict__ U,
                                                       const uint8_t* __restrict__ fmask,
                                                       const uint8_t* __restrict__ umask, float* __restrict__ part,
                                                       LbmParams P) {
    pdl_wait_trigger();
    const int z = blockIdx.y;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    float s_drho = 0.f, s_uz = 0.f, s_u2 = 0.f;
    bool inner = false;
    if (WY || WZ) {
        const int nq = P.g.nx / 2, q0 = blockIdx.x * blockDim.x;
        const int q1 = min(q0 + (int)blockDim.x, nq * P.g.ny) - 1;
        inner = q0 / nq >= 1 && q1 / nq <= P.g.ny - 2 && z >= 1 && z <= P.g.nz - 2;
    }
    if (inner) lbm_pair_cells<WX, false, false, S, CS>(fin, fout, F, U, fmask, umask, P, z, q, s_drho, s_uz, s_u2);
    else lbm_pair_cells<WX, WY, WZ, S, CS>(fin, fout, F, U, fmask, umask, P, z, q, s_drho, s_uz, s_u2);
    // per-warp partials for Eq. 18 and the mass / Mach checks
    warp_partials(s_drho, s_uz, s_u2, part, z);
}

// Density and velocity of the streamed populations of the current state
// (what the next pass will see), for read-out.
template <bool WX, bool WY, bool WZ, int S>
__global__ void k_moments(const typename Pop<S>::T* __restrict__ f, const long long* __restrict__ F,
                          const uint8_t* __restrict__ fmask, float* __restrict__ rho_out, float* __restrict__ U,
                          LbmParams P) {
    const int nx = P.g.nx, ny = P.g.ny;
    const long long C = P.g.ncell;
    const int z = blockIdx.y;
    const int xy = blockIdx.x * LBM_BLOCK + threadIdx.x;
    if (xy >= nx * ny) return;
    const int y = xy / nx, x = xy - y * nx;
    const long long cell = (long long)z * nx * ny + xy;
    float g[19];
    pull<WX, WY, WZ, S>(f, P, x, y, z, cell, g);
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        drho += g[i];
        jx += (float)CX(i) * g[i];
        jy += (float)CY(i) * g[i];
        jz += (float)CZ(i) * g[i];
    }
    drho += P.dr0;
    float Fx = P.body[0], Fy = P.body[1], Fz = P.body[2];
    if (fmask[tile_of(P.g, x, y, z)]) {
        Fx += force_value(F[cell]);
        Fy += force_value(F[C + cell]);
        Fz += force_value(F[2 * C + cell]);
    }
    const float rho = P.rho0 + drho;
    rho_out[cell] = rho;
    U[cell] = (jx + 0.5f * Fx) / rho;
    U[C + cell] = (jy + 0.5f * Fy) / rho;
    U[2 * C + cell] = (jz + 0.5f * Fz) / rho;
}

template <int S>
__global__ void k_lbm_init(typename Pop<S>::T* __restrict__ f, float* __restrict__ U, LbmParams P, float ux, float uy,
                           float uz) {
    const long long C = P.g.ncell;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const float usq = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const float cu = (float)CX(i) * ux + (float)CY(i) * uy + (float)CZ(i) * uz;
        f[(long long)i * C + c] =
            Pop<S>::cv(wgt(i) * (P.rho0 * (3.f * cu + 4.5f * cu * cu - 1.5f * usq)) + P.dw[wclass(i)]);
    }
    U[c] = ux;
    U[C + c] = uy;
    U[2 * C + c] = uz;
}

// Populations i0..i1-1 to float: mode +1 f = g + s_i, mode 0 f - w_i rho0 = g - dw_i.
template <int S>
__global__ void k_export(const typename Pop<S>::T* __restrict__ in, float* __restrict__ out, LbmParams P, int i0,
                         int i1, int mode) {
    const long long C = P.g.ncell;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    for (int i = i0; i < i1; ++i) {
        const int k = i == 0 ? 0 : (i < 7 ? 1 : 2);
        const float w = k == 0 ? 1.f / 3.f : (k == 1 ? 1.f / 18.f : 1.f / 36.f);
        const float v = Pop<S>::raw(in[(long long)i * C + c]);
        out[(long long)(i - i0) * C + c] = mode > 0 ? v + w * P.rho0 : v - P.dw[k];
    }
}

// Float populations i0..i1-1 (f) into the stored deviations g = f - s_i.
template <int S>
__global__ void k_import(const float* __restrict__ in, typename Pop<S>::T* __restrict__ out, LbmParams P, int i0,
                         int i1) {
    const long long C = P.g.ncell;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    for (int i = i0; i < i1; ++i) {
        const float w = i == 0 ? 1.f / 3.f : (i < 7 ? 1.f / 18.f : 1.f / 36.f);
        out[(long long)i * C + c] = Pop<S>::cv(in[(long long)(i - i0) * C + c] - w * P.rho0);
    }
}

// Tiles whose velocity the filament advance may read: every tile touched by
// the cells floor(s)-1 .. floor(s)+2 on each axis (the RK stages move a point
// by less than one cell, which the advance checks).
__global__ void k_mark_umask(Grid g, const double* __restrict__ pos, const int* __restrict__ counters, int cap,
                             uint8_t* __restrict__ umask) {
    pdl_wait_trigger();
    const int N = counters[CNT_N];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    mark_velocity_tiles(g, pos[i], pos[(long long)cap + i], pos[2LL * cap + i], umask);
}

// Zero the force grid in every tile the last spreading touched, then clear the tile flag.
__global__ void k_zero_force(Grid g, long long* __restrict__ F, uint8_t* __restrict__ fmask) {
    pdl_wait_trigger();
    const int t = blockIdx.x;
    if (!fmask[t]) return;
    const int tx = t % g.tnx, ty = (t / g.tnx) % g.tny, tz = t / (g.tnx * g.tny);
    for (int k = threadIdx.x; k < 512; k += blockDim.x) {
        const int x = (tx << TILE_SHIFT) + (k & 7), y = (ty << TILE_SHIFT) + ((k >> 3) & 7),
                  z = (tz << TILE_SHIFT) + (k >> 6);
        if (x < g.nx && y < g.ny && z < g.nz) {
            const long long c = ((long long)z * g.ny + y) * g.nx + x;
            F[c] = 0;
            F[g.ncell + c] = 0;
            F[2 * g.ncell + c] = 0;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) fmask[t] = 0;
}

// Force grid to and from float [3][C] (field export and import).
__global__ void k_force_export(const long long* __restrict__ F, float* __restrict__ out, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        out[k] = force_value(F[k]);
}

__global__ void k_force_import(const float* __restrict__ in, long long* __restrict__ F, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        F[k] = force_fixed(in[k]);
}

template <bool WX, bool WY, bool WZ, bool CS>
void lbm_launch(const LbmParams& P, dim3 grid, const void* fin, void* fout, const long long* F, float* U,
                const uint8_t* fmask, const uint8_t* umask, float* part, cudaStream_t s) {
    if (P.storage == STORE_F16)
        launch_pdl(k_lbm_step<WX, WY, WZ, STORE_F16, CS>, grid, P.block, 0, s, (const __half*)fin, (__half*)fout, F, U,
                   fmask, umask, part, P);
    else if (P.storage == STORE_BF16)
        launch_pdl(k_lbm_step<WX, WY, WZ, STORE_BF16, CS>, grid, P.block, 0, s, (const __nv_bfloat16*)fin,
                   (__nv_bfloat16*)fout, F, U, fmask, umask, part, P);
    else
        launch_pdl(k_lbm_step<WX, WY, WZ, STORE_F32, CS>, grid, P.block, 0, s, (const float*)fin, (float*)fout, F, U,
                   fmask, umask, part, P);
}

template <bool WX, bool WY, bool WZ>
void lbm_dispatch(const LbmParams& P, const void* fin, void* fout, const long long* F, float* U, const uint8_t* fmask,
                  const uint8_t* umask, float* part, cudaStream_t s) {
    const int nxy = P.g.nx * P.g.ny;
    if (P.storage != STORE_F32 && P.vec == 2) {
        dim3 grid((nxy / 2 + 127) / 128, P.g.nz);
        if (P.storage == STORE_F16) {
            if (P.stream_hint)
                launch_pdl(k_lbm_step_pair<WX, WY, WZ, STORE_F16, true>, grid, 128, 0, s, (const __half*)fin,
                           (__half*)fout, F, U, fmask, umask, part, P);
            else
                launch_pdl(k_lbm_step_pair<WX, WY, WZ, STORE_F16, false>, grid, 128, 0, s, (const __half*)fin,
                           (__half*)fout, F, U, fmask, umask, part, P);
        } else {
            if (P.stream_hint)
                launch_pdl(k_lbm_step_pair<WX, WY, WZ, STORE_BF16, true>, grid, 128, 0, s,
                           (const __nv_bfloat16*)fin, (__nv_bfloat16*)fout, F, U, fmask, umask, part, P);
            else
                launch_pdl(k_lbm_step_pair<WX, WY, WZ, STORE_BF16, false>, grid, 128, 0, s,
                           (const __nv_bfloat16*)fin, (__nv_bfloat16*)fout, F, U, fmask, umask, part, P);
        }
        return;
    }
    if (P.storage == STORE_F32 && (P.vec == 4 || P.vec == 2)) {
        const int groups = nxy / P.vec;
        dim3 grid((groups + 127) / 128, P.g.nz);
        if (P.vec == 4)
            launch_pdl(k_lbm_step_vec<WX, WY, WZ, 4>, grid, 128, 0, s, (const float*)fin, (float*)fout, F, U, fmask, umask,
                                                                part, P);
        else
            launch_pdl(k_lbm_step_vec<WX, WY, WZ, 2>, grid, 128, 0, s, (const float*)fin, (float*)fout, F, U, fmask, umask,
                                                                part, P);
        return;
    }
    dim3 grid((nxy + P.block - 1) / P.block, P.g.nz);
    if (P.stream_hint)
        lbm_launch<WX, WY, WZ, true>(P, grid, fin, fout, F, U, fmask, umask, part, s);
    else
        lbm_launch<WX, WY, WZ, false>(P, grid, fin, fout, F, U, fmask, umask, part, s);
}

template <bool WX, bool WY, bool WZ>
void moments_dispatch(const LbmParams& P, const void* f, const long long* F, const uint8_t* fmask, float* rho, float* U,
                      cudaStream_t s) {
    const int bpp = (P.g.nx * P.g.ny + LBM_BLOCK - 1) / LBM_BLOCK;
    dim3 grid(bpp, P.g.nz);
    if (P.storage == STORE_F16)
        k_moments<WX, WY, WZ, STORE_F16><<<grid, LBM_BLOCK, 0, s>>>((const __half*)f, F, fmask, rho, U, P);
    else if (P.storage == STORE_BF16)
        k_moments<WX, WY, WZ, STORE_BF16><<<grid, LBM_BLOCK, 0, s>>>((const __nv_bfloat16*)f, F, fmask, rho, U, P);
    else
        k_moments<WX, WY, WZ, STORE_F32><<<grid, LBM_BLOCK, 0, s>>>((const float*)f, F, fmask, rho, U, P);
}

}  // namespace

#define VLB_WALL_DISPATCH(FN, ...)                                                   \
    do {                                                                             \
        const int code = (P.g.wall[0] ? 1 : 0) | (P.g.wall[1] ? 2 : 0) | (P.g.wall[2] ? 4 : 0); \
        switch (code) {                                                              \
            case 0: FN<false, false, false>(__VA_ARGS__); break;                     \
            case 1: FN<true, false, false>(__VA_ARGS__); break;                      \
            case 2: FN<false, true, false>(__VA_ARGS__); break;                      \
            case 3: FN<true, true, false>(__VA_ARGS__); break;                       \
            case 4: FN<false, false, true>(__VA_ARGS__); break;                      \
            case 5: FN<true, false, true>(__VA_ARGS__); break;                       \
            case 6: FN<false, true, true>(__VA_ARGS__); break;                       \
            default: FN<true, true, true>(__VA_ARGS__); break;                       \
        }                                                                            \
    } while (0)

void launch_lbm_step(const LbmParams& P, const void* fin, void* fout, const long long* F, float* U,
                     const uint8_t* fmask, const uint8_t* umask, float* part, cudaStream_t s) {
    VLB_WALL_DISPATCH(lbm_dispatch, P, fin, fout, F, U, fmask, umask, part, s);
}

void launch_moments(const LbmParams& P, const void* f, const long long* F, const uint8_t* fmask, float* rho, float* U,
                    cudaStream_t s) {
    VLB_WALL_DISPATCH(moments_dispatch, P, f, F, fmask, rho, U, s);
}

void launch_lbm_init(const LbmParams& P, void* f, float* U, const double init_u[3], cudaStream_t s) {
    const long long C = P.g.ncell;
    const unsigned nb = (unsigned)((C + 255) / 256);
    const float ux = (float)init_u[0], uy = (float)init_u[1], uz = (float)init_u[2];
    if (P.storage == STORE_F16)
        k_lbm_init<STORE_F16><<<nb, 256, 0, s>>>((__half*)f, U, P, ux, uy, uz);
    else if (P.storage == STORE_BF16)
        k_lbm_init<STORE_BF16><<<nb, 256, 0, s>>>((__nv_bfloat16*)f, U, P, ux, uy, uz);
    else
        k_lbm_init<STORE_F32><<<nb, 256, 0, s>>>((float*)f, U, P, ux, uy, uz);
}

void launch_export(const LbmParams& P, const void* f, float* out, int i0, int i1, int mode, cudaStream_t s) {
    const unsigned nb = (unsigned)((P.g.ncell + 255) / 256);
    if (P.storage == STORE_F16)
        k_export<STORE_F16><<<nb, 256, 0, s>>>((const __half*)f, out, P, i0, i1, mode);
    else if (P.storage == STORE_BF16)
        k_export<STORE_BF16><<<nb, 256, 0, s>>>((const __nv_bfloat16*)f, out, P, i0, i1, mode);
    else
        k_export<STORE_F32><<<nb, 256, 0, s>>>((const float*)f, out, P, i0, i1, mode);
}

void launch_import(const LbmParams& P, const float* in, void* f, int i0, int i1, cudaStream_t s) {
    const unsigned nb = (unsigned)((P.g.ncell + 255) / 256);
    if (P.storage == STORE_F16)
        k_import<STORE_F16><<<nb, 256, 0, s>>>(in, (__half*)f, P, i0, i1);
    else if (P.storage == STORE_BF16)
        k_import<STORE_BF16><<<nb, 256, 0, s>>>(in, (__nv_bfloat16*)f, P, i0, i1);
    else
        k_import<STORE_F32><<<nb, 256, 0, s>>>(in, (float*)f, P, i0, i1);
}

int lbm_blocks_per_plane(const LbmParams& P) {
    const int nxy = P.g.nx * P.g.ny;
    if (P.vec == 4 || P.vec == 2) return (nxy / P.vec + 127) / 128;
    return (nxy + P.block - 1) / P.block;
}

int lbm_warps_per_plane(const LbmParams& P) {
    return lbm_blocks_per_plane(P) * ((P.vec == 4 || P.vec == 2) ? 128 : P.block) / 32;
}

void launch_plane_vs(const LbmParams& P, const float* part, long long* F, uint8_t* umask, uint8_t* fmask,
                     cudaStream_t s) {
    const int wpp = lbm_warps_per_plane(P);
    const int ntiles = P.g.tnx * P.g.tny * P.g.tnz, nplane = (P.g.nz + 7) / 8;
    const int nblk = std::max(nplane, std::min((ntiles + 7) / 8, 1216));  // at most 8 blocks per SM of 152
    launch_pdl(k_plane_vs, nblk, 256, 0, s, part, wpp, P, F, umask, fmask, ntiles, nplane);
}

void launch_mark_umask(const Grid& g, const double* pos, const int* counters, int cap, uint8_t* umask,
                       cudaStream_t s) {
    if (cap <= 0) return;
    launch_pdl(k_mark_umask, (cap + 127) / 128, 128, 0, s, g, pos, counters, cap, umask);
}

void launch_force_export(const Grid& g, const long long* F, float* out, cudaStream_t s) {
    k_force_export<<<1216, 256, 0, s>>>(F, out, 3 * g.ncell);
}

void launch_force_import(const Grid& g, const float* in, long long* F, cudaStream_t s) {
    k_force_import<<<1216, 256, 0, s>>>(in, F, 3 * g.ncell);
}

void launch_zero_force(const Grid& g, long long* F, uint8_t* fmask, cudaStream_t s) {
    const int ntiles = g.tnx * g.tny * g.tnz;
    launch_pdl(k_zero_force, ntiles, 256, 0, s, g, F, fmask);
}

}  // namespace vlb
