// Lattice-Boltzmann part of the coupled step (Sec. II.B of arXiv 2108.04435):
// D3Q19 BGK pull stream-collide with the split forcing of Eq. 14a-d, halfway
// bounce-back walls, moving-wall heater links (Sec. IV), the per-plane sums
// behind Eq. 18, and the activity masks that keep force/velocity traffic to
// the tiles near filaments.
//
// Populations are stored as shifted deviations g_i = f_i - w_i rho0 in FP32;
// the arithmetic below is the paper's with f_i = g_i + w_i rho0 substituted,
// which keeps the O(u) signal of each population far above FP32 rounding.
#include <cuda_runtime.h>
#include <math.h>

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

__device__ __forceinline__ int tile_of(const Grid& g, int x, int y, int z) {
    return ((z >> TILE_SHIFT) * g.tny + (y >> TILE_SHIFT)) * g.tnx + (x >> TILE_SHIFT);
}

// Pull the 19 shifted populations arriving at (x, y, z) (Eq. 14d in pull
// form).  A link whose source lies beyond a wall is bounced back half-way; on
// the z faces the moving-wall term 2 w_i rho0 (c_i . u_w)/c_s^2 with
// u_w = heater e_z injects (low face) or removes (high face) normal fluid.
template <bool WX, bool WY, bool WZ>
__device__ __forceinline__ void pull(const float* __restrict__ f, const LbmParams& P, int x, int y, int z,
                                     long long cell, float g[19]) {
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
            g[i] = __ldg(&f[(long long)i * C + ((long long)sz * ny + sy) * nx + sx]);
        } else {
            float v = __ldg(&f[(long long)opp(i) * C + cell]);
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

// K1: one lattice pass.  One thread per cell, one block per 256 consecutive
// (x, y) cells of one z plane, so every population array is read in coalesced
// rows (the +-x shift of the pull is absorbed by L1) and written aligned.
template <bool WX, bool WY, bool WZ>
__global__ void __launch_bounds__(LBM_BLOCK) k_lbm_step(const float* __restrict__ fin, float* __restrict__ fout,
                                                        const float* __restrict__ F, float* __restrict__ U,
                                                        const uint8_t* __restrict__ fmask,
                                                        const uint8_t* __restrict__ umask, double* __restrict__ part,
                                                        LbmParams P) {
    const int nx = P.g.nx, ny = P.g.ny;
    const long long C = P.g.ncell;
    const int z = blockIdx.y;
    const int xy = blockIdx.x * LBM_BLOCK + threadIdx.x;
    float s_drho = 0.f, s_uz = 0.f, s_u2 = 0.f;
    if (xy < nx * ny) {
        const int y = xy / nx, x = xy - y * nx;
        const long long cell = (long long)z * nx * ny + xy;
        float g[19];
        pull<WX, WY, WZ>(fin, P, x, y, z, cell, g);
        // Eqs. 5-6 with the half-force shift: rho = rho0 + sum g, j = sum c g
        float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            drho += g[i];
            if (CX(i)) jx += (float)CX(i) * g[i];
            if (CY(i)) jy += (float)CY(i) * g[i];
            if (CZ(i)) jz += (float)CZ(i) * g[i];
        }
        drho += P.dr0;
        const int tile = tile_of(P.g, x, y, z);
        const bool factive = fmask[tile] != 0;
        float Fx = P.body[0], Fy = P.body[1], Fz = P.body[2];
        if (factive) {
            Fx += __ldg(&F[cell]);
            Fy += __ldg(&F[C + cell]);
            Fz += __ldg(&F[2 * C + cell]);
        }
        const bool force = factive || P.body_on;
        const float rho = P.rho0 + drho;
        const float inv = 1.f / rho;
        const float ux = (jx + 0.5f * Fx) * inv, uy = (jy + 0.5f * Fy) * inv, uz = (jz + 0.5f * Fz) * inv;
        const float usq = ux * ux + uy * uy + uz * uz;
        if (umask[tile]) {
            U[cell] = ux;
            U[C + cell] = uy;
            U[2 * C + cell] = uz;
        }
        const float uF = ux * Fx + uy * Fy + uz * Fz;
        const bool pinned = P.pin_on && z == 0;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const float cu = (float)CX(i) * ux + (float)CY(i) * uy + (float)CZ(i) * uz;
            // Eq. 7 minus w_i rho0
            const float geq = wgt(i) * (drho + rho * (3.f * cu + 4.5f * cu * cu - 1.5f * usq)) + P.dw[wclass(i)];
            // Eq. 14b: BGK relaxation (Eq. 8) of the streamed population
            float out = g[i] - P.omega * (g[i] - geq);
            if (force) {
                // Eq. 13 (e_i read as c_i), applied as two halves (Eqs. 14a, 14c)
                const float cF = (float)CX(i) * Fx + (float)CY(i) * Fy + (float)CZ(i) * Fz;
                out += P.pref * wgt(i) * (3.f * (cF - uF) + 9.f * cu * cF);
            }
            if (pinned) {
                const float cp = (float)CZ(i) * P.pin;
                out = wgt(i) * (drho + rho * (3.f * cp + 4.5f * cp * cp - 1.5f * P.pin * P.pin)) + P.dw[wclass(i)];
            }
            fout[(long long)i * C + cell] = out;
        }
        s_drho = drho;
        s_uz = uz;
        s_u2 = (usq == usq) ? usq : INFINITY;
    }
    // per-block partials for Eq. 18 and the mass / Mach checks
    __shared__ double red[3][LBM_BLOCK / 32];
    s_drho = warp_reduce<0>(s_drho);
    s_uz = warp_reduce<0>(s_uz);
    s_u2 = warp_reduce<1>(s_u2);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = s_drho;
        red[1][wid] = s_uz;
        red[2][wid] = s_u2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, m = 0.0;
#pragma unroll
        for (int w = 0; w < LBM_BLOCK / 32; ++w) {
            a += red[0][w];
            b += red[1][w];
            m = fmax(m, red[2][w]);
        }
        double* o = part + ((long long)z * gridDim.x + blockIdx.x) * 3;
        o[0] = a;
        o[1] = b;
        o[2] = m;
    }
}

// Density and velocity of the streamed populations of the current state
// (what the next pass will see), for read-out.
template <bool WX, bool WY, bool WZ>
__global__ void k_moments(const float* __restrict__ f, const float* __restrict__ F, const uint8_t* __restrict__ fmask,
                          float* __restrict__ rho_out, float* __restrict__ U, LbmParams P) {
    const int nx = P.g.nx, ny = P.g.ny;
    const long long C = P.g.ncell;
    const int z = blockIdx.y;
    const int xy = blockIdx.x * LBM_BLOCK + threadIdx.x;
    if (xy >= nx * ny) return;
    const int y = xy / nx, x = xy - y * nx;
    const long long cell = (long long)z * nx * ny + xy;
    float g[19];
    pull<WX, WY, WZ>(f, P, x, y, z, cell, g);
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
        Fx += F[cell];
        Fy += F[C + cell];
        Fz += F[2 * C + cell];
    }
    const float rho = P.rho0 + drho;
    rho_out[cell] = rho;
    U[cell] = (jx + 0.5f * Fx) / rho;
    U[C + cell] = (jy + 0.5f * Fy) / rho;
    U[2 * C + cell] = (jz + 0.5f * Fz) / rho;
}

__global__ void k_lbm_init(float* __restrict__ f, float* __restrict__ U, LbmParams P, float ux, float uy, float uz) {
    const long long C = P.g.ncell;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const float usq = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const float cu = (float)CX(i) * ux + (float)CY(i) * uy + (float)CZ(i) * uz;
        f[(long long)i * C + c] = wgt(i) * (P.rho0 * (3.f * cu + 4.5f * cu * cu - 1.5f * usq)) + P.dw[wclass(i)];
    }
    U[c] = ux;
    U[C + c] = uy;
    U[2 * C + c] = uz;
}

// direction +1: out = g + w_i rho0 (export); -1: out = f - w_i rho0 (import)
__global__ void k_unshift(const float* __restrict__ in, float* __restrict__ out, LbmParams P, int direction) {
    const long long C = P.g.ncell;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const float s = wgt(i) * P.rho0;
        out[(long long)i * C + c] = direction > 0 ? in[(long long)i * C + c] + s : in[(long long)i * C + c] - s;
    }
}

// Eq. 18 per z plane from the block partials, in a fixed order; mass and the
// Mach limit of Sec. II.B (|u|/c_s < 0.05) are checked here as well.
__global__ void k_plane_vs(const double* __restrict__ part, int nz, int bpp, double area, double ncell, double rho0,
                           double inv_ratio, int periodic, double* __restrict__ Vs, double* __restrict__ dstats,
                           int* __restrict__ counters) {
    __shared__ double s_tot[256], s_mass[256], s_max[256];
    double tot = 0.0, mass = 0.0, mx = 0.0;
    for (int p = threadIdx.x; p < nz; p += blockDim.x) {
        double su = 0.0, sr = 0.0, m = 0.0;
        for (int b = 0; b < bpp; ++b) {
            const double* o = part + ((long long)p * bpp + b) * 3;
            sr += o[0];
            su += o[1];
            m = fmax(m, o[2]);
        }
        if (!periodic) Vs[p] = -inv_ratio * (su / area);
        tot += su;
        mass += sr;
        mx = fmax(mx, m);
    }
    s_tot[threadIdx.x] = tot;
    s_mass[threadIdx.x] = mass;
    s_max[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s_tot[threadIdx.x] += s_tot[threadIdx.x + o];
            s_mass[threadIdx.x] += s_mass[threadIdx.x + o];
            s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (periodic) {
        const double v = -inv_ratio * (s_tot[0] / ncell);
        for (int p = threadIdx.x; p < nz; p += blockDim.x) Vs[p] = v;
    }
    if (threadIdx.x == 0) {
        const double m = s_max[0];
        const double mach = sqrt(3.0 * m);
        dstats[DS_MASS] = rho0 * ncell + s_mass[0];
        dstats[DS_MAXMACH] = mach;
        int st = 0;
        if (!(mach < 0.05)) st |= ST_MACH;
        if (!isfinite(m) || !isfinite(s_mass[0])) st |= ST_NAN;
        if (st) atomicOr(&counters[CNT_STATUS], st);
    }
}

// Tiles whose velocity the filament advance may read: every tile touched by
// the cells floor(s)-1 .. floor(s)+2 on each axis (the RK stages move a point
// by less than one cell, which the advance checks).
__global__ void k_mark_umask(Grid g, const double* __restrict__ pos, const int* __restrict__ counters, int cap,
                             uint8_t* __restrict__ umask) {
    const int N = counters[CNT_N];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int n[3] = {g.nx, g.ny, g.nz};
    int t[3][4];
    for (int a = 0; a < 3; ++a) {
        const int b = (int)floor(pos[(long long)a * cap + i]);
        for (int k = 0; k < 4; ++k) {
            int c = b - 1 + k;
            if (g.wall[a]) c = c < 0 ? 0 : (c > n[a] - 1 ? n[a] - 1 : c);
            else c = ((c % n[a]) + n[a]) % n[a];
            t[a][k] = c >> TILE_SHIFT;
        }
    }
    for (int kz = 0; kz < 4; ++kz)
        for (int ky = 0; ky < 4; ++ky)
            for (int kx = 0; kx < 4; ++kx) umask[(t[2][kz] * g.tny + t[1][ky]) * g.tnx + t[0][kx]] = 1;
}

// Zero the force grid in every tile the last spreading touched, then clear the tile flag.
__global__ void k_zero_force(Grid g, float* __restrict__ F, uint8_t* __restrict__ fmask) {
    const int t = blockIdx.x;
    if (!fmask[t]) return;
    const int tx = t % g.tnx, ty = (t / g.tnx) % g.tny, tz = t / (g.tnx * g.tny);
    for (int k = threadIdx.x; k < 512; k += blockDim.x) {
        const int x = (tx << TILE_SHIFT) + (k & 7), y = (ty << TILE_SHIFT) + ((k >> 3) & 7),
                  z = (tz << TILE_SHIFT) + (k >> 6);
        if (x < g.nx && y < g.ny && z < g.nz) {
            const long long c = ((long long)z * g.ny + y) * g.nx + x;
            F[c] = 0.f;
            F[g.ncell + c] = 0.f;
            F[2 * g.ncell + c] = 0.f;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) fmask[t] = 0;
}

template <bool WX, bool WY, bool WZ>
void lbm_dispatch(const LbmParams& P, const float* fin, float* fout, const float* F, float* U, const uint8_t* fmask,
                  const uint8_t* umask, double* part, cudaStream_t s) {
    const int bpp = (P.g.nx * P.g.ny + LBM_BLOCK - 1) / LBM_BLOCK;
    dim3 grid(bpp, P.g.nz);
    k_lbm_step<WX, WY, WZ><<<grid, LBM_BLOCK, 0, s>>>(fin, fout, F, U, fmask, umask, part, P);
}

template <bool WX, bool WY, bool WZ>
void moments_dispatch(const LbmParams& P, const float* f, const float* F, const uint8_t* fmask, float* rho, float* U,
                      cudaStream_t s) {
    const int bpp = (P.g.nx * P.g.ny + LBM_BLOCK - 1) / LBM_BLOCK;
    dim3 grid(bpp, P.g.nz);
    k_moments<WX, WY, WZ><<<grid, LBM_BLOCK, 0, s>>>(f, F, fmask, rho, U, P);
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

void launch_lbm_step(const LbmParams& P, const float* fin, float* fout, const float* F, float* U,
                     const uint8_t* fmask, const uint8_t* umask, double* part, cudaStream_t s) {
    VLB_WALL_DISPATCH(lbm_dispatch, P, fin, fout, F, U, fmask, umask, part, s);
}

void launch_moments(const LbmParams& P, const float* f, const float* F, const uint8_t* fmask, float* rho, float* U,
                    cudaStream_t s) {
    VLB_WALL_DISPATCH(moments_dispatch, P, f, F, fmask, rho, U, s);
}

void launch_lbm_init(const LbmParams& P, float* f, float* U, const double init_u[3], cudaStream_t s) {
    const long long C = P.g.ncell;
    k_lbm_init<<<(unsigned)((C + 255) / 256), 256, 0, s>>>(f, U, P, (float)init_u[0], (float)init_u[1],
                                                           (float)init_u[2]);
}

void launch_unshift(const LbmParams& P, const float* in, float* out, int direction, cudaStream_t s) {
    const long long C = P.g.ncell;
    k_unshift<<<(unsigned)((C + 255) / 256), 256, 0, s>>>(in, out, P, direction);
}

void launch_plane_vs(const LbmParams& P, const double* part, double ratio, double* Vs, double* dstats, int* counters,
                     cudaStream_t s) {
    const int bpp = (P.g.nx * P.g.ny + LBM_BLOCK - 1) / LBM_BLOCK;
    const double area = (double)P.g.nx * (double)P.g.ny;
    k_plane_vs<<<1, 256, 0, s>>>(part, P.g.nz, bpp, area, (double)P.g.ncell, (double)P.rho0, 1.0 / ratio,
                                 P.g.wall[2] ? 0 : 1, Vs, dstats, counters);
}

void launch_mark_umask(const Grid& g, const double* pos, const int* counters, int cap, uint8_t* umask,
                       cudaStream_t s) {
    if (cap <= 0) return;
    k_mark_umask<<<(cap + 127) / 128, 128, 0, s>>>(g, pos, counters, cap, umask);
}

void launch_zero_force(const Grid& g, float* F, uint8_t* fmask, cudaStream_t s) {
    const int ntiles = g.tnx * g.tny * g.tnz;
    k_zero_force<<<ntiles, 256, 0, s>>>(g, F, fmask);
}

}  // namespace vlb
