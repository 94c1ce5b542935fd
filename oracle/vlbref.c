/*
 * vlbref.c -- plain FP64 CPU oracle of the coupled VFM-LBM step of
 * Inui & Tsubota, arXiv 2108.04435 (Sec. II).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It is deliberately
 * slow and literal: every loop follows one equation of the paper, in the
 * paper's order, in IEEE double precision with no FMA contraction
 * (build with -ffp-contract=off).  OpenMP only parallelises loops whose
 * iterations are independent, so results do not depend on the thread count.
 *
 * Where the paper is silent the readings below are used (all listed in the
 * design notes of the repository):
 *  - u carries the half-force shift u = (sum c f + F/2)/rho in f^eq, in F_i and
 *    as the normal-fluid velocity seen by the vortices (Eq. 6 with Guo's shift,
 *    implied by the (1 - 1/2tau) prefactor of Eq. 13).
 *  - e_i of Eq. 13 is read as c_i.
 *  - walls: halfway bounce-back; the heater faces of the stream axis are
 *    moving-wall (Ladd) links carrying u_w = heater_vn e_s (Sec. IV).
 *  - V_s per stream plane from Eq. 18 (plain plane mean of u); a periodic
 *    stream axis uses the box mean.
 *  - Biot-Savart: exact line integral of Eq. 3 over straight segments, minimum
 *    image on periodic axes, the two segments touching the target excluded and
 *    replaced by the local term beta s' x s'' with Schwarz's cutoff
 *    beta = kappa/(4 pi) ln(2 sqrt(l+ l-)/(e^{1/4} a)).
 *  - Wall images (wall_images = 1): v_s,b from first-order mirror images of
 *    every segment across each solid wall face, orientation reversed; a pinned
 *    end skips the image of its own segment across its own wall (image_velocity()).
 *  - Time integration: classic RK4 over one lattice step (or vfm_substeps
 *    sub-steps) with u, V_s frozen; the reaction of Eq. 10 is taken from the
 *    first stage and spread with the 2-point delta function of Eq. 11.  The
 *    force grid is the force of the next lattice pass only, which consumes it.
 *  - Remeshing and reconnection rules (Sec. II.A only fixes the resolution
 *    [dxi_min, dxi_max] and "exchange legs within the resolution"): see
 *    remesh() and reconnect() below.
 *
 * Stats array (VLBREF_FIELD_STATS, 16 doubles):
 *   0 points  1 status bits  2 mass  3 line length  4 max Mach  5 splits
 *   6 merges  7 reconnections  8 points deleted in small loops  9 steps
 *   10..12 momentum sum(rho u)  13 wall-contact cuts  14..15 reserved
 * Status bits: 1 Mach >= 0.05, 2 NaN, 4 capacity, 16 stage displacement >= 1.
 */
#include "vlbref.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define Q 19
#define PI 3.14159265358979323846

/* Table I: D3Q19 velocities and weights (0-based; opposite pairs adjacent). */
static const int CV[Q][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double WV[Q] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static int opposite(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

enum { ST_MACH = 1, ST_NAN = 2, ST_CAPACITY = 4, ST_CFL = 16 };

struct vlbref_channel {
    vlbref_params p;
    long ncell;
    double* f;     /* post-collision populations f*, [Q][C] */
    double* ftmp;
    double* F;     /* force grid, [3][C] */
    double* U;     /* u^n of the last LBM pass, [3][C] */
    double* RHO;   /* rho^n of the last LBM pass, [C] */
    double* Vs;    /* superfluid velocity per stream plane (Eq. 18) */
    double mass, max_mach, mom[3];
    int status;
    long steps;
    int N, cap;
    double* pos;   /* [cap][3] */
    int* next;
    int* prev;
    double* vel1;  /* [cap][3] stage-1 ds/dt of the last advance */
    long n_split, n_merge, n_reconnect, n_small, n_wallcut;
    char err[256];
};

/* ------------------------------------------------------------------ helpers */

static long cell_index(const vlbref_channel* ch, int x, int y, int z) {
    return ((long)z * ch->p.n[1] + y) * ch->p.n[0] + x;
}

/* minimum-image difference along one axis (periodic axes only) */
static double min_image(const vlbref_channel* ch, int axis, double d) {
    if (!ch->p.wall[axis]) {
        double L = (double)ch->p.n[axis];
        if (d > 0.5 * L) d -= L;
        else if (d < -0.5 * L) d += L;
    }
    return d;
}

static void diff3(const vlbref_channel* ch, const double* a, const double* b, double* out) {
    /* out = mi(a - b) */
    for (int k = 0; k < 3; ++k) out[k] = min_image(ch, k, a[k] - b[k]);
}

static double norm3(const double* a) { return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* out) {
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

static void set_err(vlbref_channel* ch, const char* msg) {
    if (ch) snprintf(ch->err, sizeof ch->err, "%s", msg);
}

/* Walls sit halfway between the last fluid node and the outside, at -1/2
 * and n - 1/2; filament points are kept dxi_min/2 inside them.  These are the
 * two clamp bounds of a wall axis. */
static double wall_lo(const vlbref_channel* ch) { return -0.5 + 0.5 * ch->p.dxi_min; }
static double wall_hi(const vlbref_channel* ch, int a) { return (double)ch->p.n[a] - 0.5 - 0.5 * ch->p.dxi_min; }

/* The first clamp bound that position s touches, in the order x-, x+, y-, y+,
 * z-, z+, as 2*axis + side (side 1 = high wall); -1 when none.  An open end of
 * a line is pinned to this wall. */
static int touching_wall(const vlbref_channel* ch, const double* s) {
    for (int a = 0; a < 3; ++a) {
        if (!ch->p.wall[a]) continue;
        if (s[a] <= wall_lo(ch)) return 2 * a;
        if (s[a] >= wall_hi(ch, a)) return 2 * a + 1;
    }
    return -1;
}

/* --------------------------------------------------------- LBM pieces (II.B) */

/* Eq. 7 with c_s^2 = 1/3 */
static double feq_i(int i, double rho, const double* u) {
    double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return WV[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

/* Eq. 13, e_i read as c_i, c_s^2 = 1/3 */
static double force_i(int i, const double* u, const double* F, double tau) {
    double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
    double cF = CV[i][0] * F[0] + CV[i][1] * F[1] + CV[i][2] * F[2];
    double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    return (1.0 - 1.0 / (2.0 * tau)) * WV[i] * (3.0 * (cF - uF) + 9.0 * cu * cF);
}

/* Streaming (Eq. 9 / 14d) in pull form: the population arriving at x along c_i.
 * A link whose source lies beyond a wall is bounced back (halfway), with the
 * moving-wall term 2 w_i rho0 (c_i . u_w)/c_s^2 on the stream-axis faces. */
static double pulled(const vlbref_channel* ch, const double* fsrc, int i, int x, int y, int z) {
    int xyz[3] = {x, y, z};
    int src[3];
    int outside = 0, stream_face = 0;
    for (int a = 0; a < 3; ++a) {
        int s = xyz[a] - CV[i][a];
        int n = ch->p.n[a];
        if (s < 0 || s >= n) {
            if (ch->p.wall[a]) {
                outside = 1;
                if (a == ch->p.stream_axis) stream_face = 1;
            } else {
                s = (s + n) % n;
            }
        }
        src[a] = s;
    }
    if (!outside) return fsrc[(long)i * ch->ncell + cell_index(ch, src[0], src[1], src[2])];
    double uw = stream_face ? ch->p.heater_vn : 0.0;
    double cuw = CV[i][ch->p.stream_axis] * uw;
    return fsrc[(long)opposite(i) * ch->ncell + cell_index(ch, x, y, z)] + 2.0 * WV[i] * ch->p.rho0 * cuw * 3.0;
}

/* Moments of the pulled populations (Eqs. 5-6 with the half-force shift). */
static void moments(const vlbref_channel* ch, const double* fin, long c, double* rho, double* u, double* Ftot) {
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
        r += fin[i];
        for (int a = 0; a < 3; ++a) j[a] += CV[i][a] * fin[i];
    }
    for (int a = 0; a < 3; ++a) {
        Ftot[a] = ch->F[(long)a * ch->ncell + c] + ch->p.body_force[a];
        u[a] = (j[a] + 0.5 * Ftot[a]) / r;
    }
    *rho = r;
}

/* One LBM pass: Eq. 14a-d in pull form, then Eq. 18 per plane. */
static void lbm_pass(vlbref_channel* ch) {
    const int nx = ch->p.n[0], ny = ch->p.n[1], nz = ch->p.n[2];
    const double tau = ch->p.tau;
    const int sa = ch->p.stream_axis;
    const long C = ch->ncell;
#pragma omp parallel for schedule(static)
    for (long row = 0; row < (long)ny * nz; ++row) {
        int y = (int)(row % ny), z = (int)(row / ny);
        for (int x = 0; x < nx; ++x) {
            long c = cell_index(ch, x, y, z);
            double fin[Q], rho, u[3], Ft[3];
            for (int i = 0; i < Q; ++i) fin[i] = pulled(ch, ch->f, i, x, y, z);
            moments(ch, fin, c, &rho, u, Ft);
            int xyz[3] = {x, y, z};
            int pinned = (ch->p.pin_vn != 0.0) && !ch->p.wall[sa] && xyz[sa] == 0;
            double upin[3] = {0.0, 0.0, 0.0};
            upin[sa] = ch->p.pin_vn;
            for (int i = 0; i < Q; ++i) {
                double feq = feq_i(i, rho, u);
                double Fi = force_i(i, u, Ft, tau);
                double f1 = fin[i] + 0.5 * Fi;            /* Eq. 14a */
                double f2 = f1 - (fin[i] - feq) / tau;    /* Eq. 14b (uses f, as printed) */
                double f3 = f2 + 0.5 * Fi;                /* Eq. 14c */
                if (pinned) f3 = feq_i(i, rho, upin);     /* counterflow pinned plane (Sec. III.C) */
                ch->ftmp[(long)i * C + c] = f3;           /* stored for the pull of Eq. 14d */
            }
            for (int a = 0; a < 3; ++a) ch->U[(long)a * C + c] = u[a];
            ch->RHO[c] = rho;
        }
    }
    double* t = ch->f; ch->f = ch->ftmp; ch->ftmp = t;

    /* Eq. 18: V_s(plane) = -(rho_n/rho_s) * plane mean of u_s */
    const int ns = ch->p.n[sa];
    double* psum = (double*)calloc((size_t)ns, sizeof(double));
    double mass = 0.0, maxu2 = 0.0, mom[3] = {0.0, 0.0, 0.0};
    int nan = 0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long c = cell_index(ch, x, y, z);
                int xyz[3] = {x, y, z};
                double rho = ch->RHO[c];
                double u[3] = {ch->U[c], ch->U[C + c], ch->U[2 * C + c]};
                psum[xyz[sa]] += u[sa];
                mass += rho;
                for (int a = 0; a < 3; ++a) mom[a] += rho * u[a];
                double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                if (u2 > maxu2) maxu2 = u2;
                if (rho != rho || u2 != u2) nan = 1;
            }
    const double area = (double)C / (double)ns;
    const double rn_rs = 1.0 / ch->p.rho_s_over_rho_n;
    if (ch->p.wall[sa]) {
        for (int k = 0; k < ns; ++k) ch->Vs[k] = -rn_rs * (psum[k] / area);
    } else {
        double tot = 0.0;
        for (int k = 0; k < ns; ++k) tot += psum[k];
        for (int k = 0; k < ns; ++k) ch->Vs[k] = -rn_rs * (tot / (double)C);
    }
    free(psum);
    ch->mass = mass;
    for (int a = 0; a < 3; ++a) ch->mom[a] = mom[a];
    ch->max_mach = sqrt(3.0 * maxu2);
    if (ch->max_mach >= 0.05) ch->status |= ST_MACH; /* Sec. II.B: |u|/c_s < 0.05 */
    if (nan) ch->status |= ST_NAN;
    /* The force grid holds the friction reaction for this one lattice pass
     * (the reaction spread in step n acts in the next lattice step only): the
     * pass consumes it. */
    memset(ch->F, 0, sizeof(double) * 3 * (size_t)C);
}

/* -------------------------------------------- coupling: Eq. 11 (2-point delta) */

/* Node indices and 1-D weights of delta_2pt around coordinate s on one axis.
 * Periodic axes wrap; on wall axes a node beyond the fluid is replaced by the
 * nearest fluid node (its weight moves there, the weights still sum to 1). */
static void delta_axis(const vlbref_channel* ch, int axis, double s, int* i0, int* i1, double* w0, double* w1) {
    double fl = floor(s);
    int b = (int)fl;
    double fr = s - fl;
    *w0 = 1.0 - fr;
    *w1 = fr;
    int n = ch->p.n[axis];
    int a0 = b, a1 = b + 1;
    if (!ch->p.wall[axis]) {
        a0 = ((a0 % n) + n) % n;
        a1 = ((a1 % n) + n) % n;
    } else {
        if (a0 < 0) a0 = 0;
        if (a0 > n - 1) a0 = n - 1;
        if (a1 < 0) a1 = 0;
        if (a1 > n - 1) a1 = n - 1;
    }
    *i0 = a0;
    *i1 = a1;
}

static void interp_u(const vlbref_channel* ch, const double* field, const double* s, double* out) {
    int ix[2], iy[2], iz[2];
    double wx[2], wy[2], wz[2];
    delta_axis(ch, 0, s[0], &ix[0], &ix[1], &wx[0], &wx[1]);
    delta_axis(ch, 1, s[1], &iy[0], &iy[1], &wy[0], &wy[1]);
    delta_axis(ch, 2, s[2], &iz[0], &iz[1], &wz[0], &wz[1]);
    out[0] = out[1] = out[2] = 0.0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                double w = wz[cz] * wy[cy] * wx[cx];
                long c = cell_index(ch, ix[cx], iy[cy], iz[cz]);
                for (int a = 0; a < 3; ++a) out[a] += w * field[(long)a * ch->ncell + c];
            }
}

static void spread_g(vlbref_channel* ch, const double* s, const double* g) {
    int ix[2], iy[2], iz[2];
    double wx[2], wy[2], wz[2];
    delta_axis(ch, 0, s[0], &ix[0], &ix[1], &wx[0], &wx[1]);
    delta_axis(ch, 1, s[1], &iy[0], &iy[1], &wy[0], &wy[1]);
    delta_axis(ch, 2, s[2], &iz[0], &iz[1], &wz[0], &wz[1]);
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                double w = wz[cz] * wy[cy] * wx[cx];
                long c = cell_index(ch, ix[cx], iy[cy], iz[cz]);
                for (int a = 0; a < 3; ++a) ch->F[(long)a * ch->ncell + c] += w * g[a];
            }
}

/* V_s of Eq. 18 at a point: the plane values under the same 1-D weights. */
static double vs_at(const vlbref_channel* ch, const double* s) {
    int sa = ch->p.stream_axis, i0, i1;
    double w0, w1;
    delta_axis(ch, sa, s[sa], &i0, &i1, &w0, &w1);
    return w0 * ch->Vs[i0] + w1 * ch->Vs[i1];
}

/* ------------------------------------------------------- VFM pieces (II.A) */

/* Exact integral of the Eq. 3 kernel over the straight segment starting at
 * R1 = s1 - r with direction d (R2 = R1 + d); adds into out. */
static void segment_add(const double* R1, const double* d, double kappa, double* out) {
    double R2[3] = {R1[0] + d[0], R1[1] + d[1], R1[2] + d[2]};
    double a = norm3(R1), b = norm3(R2);
    double ab = a * b;
    double dt = dot3(R1, R2);
    if (ab == 0.0 || ab + dt <= 1e-12 * ab) return; /* target on the segment */
    double cr[3];
    cross3(R1, R2, cr);
    double fac = kappa / (4.0 * PI) * (a + b) / (ab * (ab + dt));
    for (int k = 0; k < 3; ++k) out[k] += fac * cr[k];
}

/* Per-point geometry of the discretised filament: three-point derivatives on
 * the non-uniform arc-length grid, the segment-length weight and the local
 * (LIA) velocity beta s' x s'' of the divergent part of Eq. 3. */
/* An open end pinned on a wall takes as its missing neighbour the mirror image
 * of its present neighbour across that wall (the line continued by its image);
 * an end touching no wall (not produced by the rules below) is continued
 * straight.  The end represents half of its one real segment. */
static void point_geometry(const vlbref_channel* ch, const double* s, int i, double* sp, double* spp,
                           double* dxi, double* lia, double* lplus) {
    int p = ch->prev[i], q = ch->next[i];
    double a[3], b[3];
    if (p >= 0) diff3(ch, &s[3 * i], &s[3 * p], a); /* s_i - s_p */
    if (q >= 0) diff3(ch, &s[3 * q], &s[3 * i], b); /* s_q - s_i */
    if (p < 0 || q < 0) {
        int nb = p < 0 ? q : p, code = touching_wall(ch, &s[3 * i]);
        double g[3], *ghost_diff = p < 0 ? a : b;
        for (int k = 0; k < 3; ++k) g[k] = s[3 * nb + k];
        if (code >= 0) {
            int ax = code >> 1;
            double w = (code & 1) ? (double)ch->p.n[ax] - 0.5 : -0.5;
            g[ax] = 2.0 * w - s[3 * nb + ax];
            if (p < 0) diff3(ch, &s[3 * i], g, ghost_diff); /* s_i - ghost */
            else diff3(ch, g, &s[3 * i], ghost_diff);       /* ghost - s_i */
        } else {
            for (int k = 0; k < 3; ++k) ghost_diff[k] = p < 0 ? b[k] : a[k];
        }
    }
    double lm = norm3(a), lp = norm3(b);
    double den = lp * lm * (lp + lm);
    for (int k = 0; k < 3; ++k) {
        sp[k] = (lm * lm * b[k] + lp * lp * a[k]) / den;
        spp[k] = 2.0 * (lm * b[k] - lp * a[k]) / den;
    }
    *dxi = p < 0 ? 0.5 * lp : (q < 0 ? 0.5 * lm : 0.5 * (lp + lm));
    double beta = ch->p.kappa / (4.0 * PI) * log(2.0 * sqrt(lp * lm) / (exp(0.25) * ch->p.core_a));
    double c[3];
    cross3(sp, spp, c);
    for (int k = 0; k < 3; ++k) lia[k] = beta * c[k];
    if (lplus) *lplus = lp;
}

/* Boundary-induced velocity v_s,b (Sec. II.A) from images: each segment
 * j -> q is mirrored across each solid wall face (x_a -> 2w - x_a, walls at
 * w = -1/2 and n_a - 1/2) with its orientation reversed, i.e. the image
 * segment runs from M(s_q) to M(s_j); first-order images only.  A pinned end
 * does not see the image, across its own wall, of its one segment: that
 * image continues the line through the wall and belongs to its local term. */
static void image_velocity(const vlbref_channel* ch, const double* s, const double* seg, int i, double* out) {
    const int N = ch->N;
    int own_face = -1, own_seg = -1;
    if (ch->prev[i] < 0 || ch->next[i] < 0) {
        own_face = touching_wall(ch, &s[3 * i]);
        own_seg = ch->prev[i] < 0 ? i : ch->prev[i];
    }
    for (int a = 0; a < 3; ++a) {
        if (!ch->p.wall[a]) continue;
        for (int side = 0; side < 2; ++side) {
            const double w = side ? (double)ch->p.n[a] - 0.5 : -0.5;
            for (int j = 0; j < N; ++j) {
                const int q = ch->next[j];
                if (q < 0) continue;
                if (2 * a + side == own_face && j == own_seg) continue;
                double start[3], d[3], R1[3];
                for (int k = 0; k < 3; ++k) {
                    start[k] = s[3 * q + k];
                    d[k] = -seg[3 * j + k]; /* M(s_j) - M(s_q) off the normal axis */
                }
                start[a] = 2.0 * w - s[3 * q + a];
                d[a] = seg[3 * j + a];
                diff3(ch, start, &s[3 * i], R1);
                segment_add(R1, d, ch->p.kappa, out);
            }
        }
    }
}

/* Velocity ds/dt of every point at positions s (Eq. 3 + Eq. 4).  When
 * spread != 0, the reaction of Eq. 10 on the normal fluid is spread into F. */
static void filament_velocity(vlbref_channel* ch, const double* s, double* k, double* vbs_out, int spread) {
    const int N = ch->N;
    const int sa = ch->p.stream_axis;
    double* sp = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* spp = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* dxi = (double*)malloc(sizeof(double) * (size_t)N);
    double* lia = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* seg = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* fr = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    for (int i = 0; i < N; ++i) {
        point_geometry(ch, s, i, &sp[3 * i], &spp[3 * i], &dxi[i], &lia[3 * i], NULL);
        if (ch->next[i] >= 0) diff3(ch, &s[3 * ch->next[i]], &s[3 * i], &seg[3 * i]); /* segment i -> next(i) */
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < N; ++i) {
        double vbs[3] = {0.0, 0.0, 0.0};
        for (int j = 0; j < N; ++j) {
            if (j == i || ch->next[j] == i || ch->next[j] < 0) continue; /* adjacent: local term; open end: none */
            double R1[3];
            diff3(ch, &s[3 * j], &s[3 * i], R1);
            segment_add(R1, &seg[3 * j], ch->p.kappa, vbs);
        }
        if (ch->p.wall_images) image_velocity(ch, s, seg, i, vbs);
        double vs[3], vn[3], w[3], t[3], tt[3];
        for (int a = 0; a < 3; ++a) vs[a] = vbs[a] + lia[3 * i + a];
        vs[sa] += vs_at(ch, &s[3 * i]); /* v_s,a: counterflow superfluid velocity (Eq. 18) */
        interp_u(ch, ch->U, &s[3 * i], vn);
        for (int a = 0; a < 3; ++a) w[a] = vn[a] - vs[a];
        cross3(&sp[3 * i], w, t);  /* s' x (v_n - v_s) */
        cross3(&sp[3 * i], t, tt); /* s' x [s' x (v_n - v_s)] */
        for (int a = 0; a < 3; ++a) {
            fr[3 * i + a] = ch->p.alpha * t[a] - ch->p.alpha_p * tt[a];
            k[3 * i + a] = vs[a] + fr[3 * i + a]; /* Eq. 4 */
        }
        if (ch->prev[i] < 0 || ch->next[i] < 0) { /* a pinned end slides along its wall */
            int code = touching_wall(ch, &s[3 * i]);
            if (code >= 0) k[3 * i + (code >> 1)] = 0.0;
        }
        if (vbs_out)
            for (int a = 0; a < 3; ++a) vbs_out[3 * i + a] = vbs[a];
    }
    if (spread && ch->p.couple) {
        /* Eq. 10: f/(rho_s kappa) equals the friction part of Eq. 4; the
         * reaction -f per unit length, times the length dxi represented by the
         * point and divided by rho_n (the lattice density rho0 stands for
         * rho_n), is spread onto the lattice with Eq. 11. */
        const double gscale = -ch->p.rho_s_over_rho_n * ch->p.rho0 * ch->p.kappa;
        for (int i = 0; i < N; ++i) {
            double gv[3], g[3];
            /* form 1 reads f as the drag of the Magnus balance, f = rho_s kappa fr x s' */
            if (ch->p.force_form == 1) cross3(&fr[3 * i], &sp[3 * i], gv);
            else for (int a = 0; a < 3; ++a) gv[a] = fr[3 * i + a];
            for (int a = 0; a < 3; ++a) g[a] = gscale * dxi[i] * gv[a];
            spread_g(ch, &s[3 * i], g);
        }
    }
    free(sp); free(spp); free(dxi); free(lia); free(seg); free(fr);
}

static void wrap_or_clamp(const vlbref_channel* ch, double* s) {
    for (int a = 0; a < 3; ++a) {
        double L = (double)ch->p.n[a];
        if (!ch->p.wall[a]) {
            if (s[a] < 0.0) s[a] += L;
            else if (s[a] >= L) s[a] -= L;
        } else {
            double lo = -0.5 + 0.5 * ch->p.dxi_min, hi = L - 0.5 - 0.5 * ch->p.dxi_min;
            if (s[a] < lo) s[a] = lo;
            if (s[a] > hi) s[a] = hi;
        }
    }
}

/* Eq. 4 integrated with classic RK4 (u^n and V_s^n frozen over the step). */
static void vfm_advance(vlbref_channel* ch) {
    const int N = ch->N;
    if (N == 0) return;
    const int nsub = ch->p.vfm_substeps > 0 ? ch->p.vfm_substeps : 1;
    const double dt = 1.0 / nsub;
    size_t sz = sizeof(double) * 3 * (size_t)N;
    double* s0 = (double*)malloc(sz);
    double* st = (double*)malloc(sz);
    double* kk = (double*)malloc(sz);
    double* acc = (double*)malloc(sz);
    for (int sub = 0; sub < nsub; ++sub) {
        memcpy(s0, ch->pos, sz);
        /* zero the force grid before the reaction of this step is spread */
        if (sub == 0 && ch->p.couple) memset(ch->F, 0, sizeof(double) * 3 * (size_t)ch->ncell);
        const double cst[4] = {0.0, 0.5, 0.5, 1.0};
        const double wst[4] = {1.0, 2.0, 2.0, 1.0};
        for (int stage = 0; stage < 4; ++stage) {
            for (int m = 0; m < 3 * N; ++m) st[m] = s0[m];
            if (stage > 0)
                for (int m = 0; m < 3 * N; ++m) st[m] = s0[m] + cst[stage] * dt * kk[m];
            filament_velocity(ch, st, kk, NULL, stage == 0 && sub == 0);
            if (stage == 0 && sub == 0) memcpy(ch->vel1, kk, sz);
            for (int m = 0; m < 3 * N; ++m) {
                if (stage == 0) acc[m] = kk[m];
                else acc[m] = acc[m] + wst[stage] * kk[m];
                if (fabs(dt * kk[m]) >= 1.0) ch->status |= ST_CFL;
            }
        }
        for (int i = 0; i < N; ++i) {
            for (int a = 0; a < 3; ++a) ch->pos[3 * i + a] = s0[3 * i + a] + (dt / 6.0) * acc[3 * i + a];
            wrap_or_clamp(ch, &ch->pos[3 * i]);
        }
    }
    free(s0); free(st); free(kk); free(acc);
}

/* --------------------------------------------------------------- topology */

/* Merge priority: the 32-bit finaliser of MurmurHash3 (fmix32) applied to the
 * point index; a candidate is removed only if no candidate neighbour outranks it. */
static uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

static int outranks(int a, int b) {
    uint32_t ha = fmix32((uint32_t)a), hb = fmix32((uint32_t)b);
    return ha > hb || (ha == hb && a < b);
}

/* Is point i on a loop or an open line of fewer than five points?  prev must
 * be the predecessor array of next (-1 at a line's first point). */
static int in_small_component(const int* next, const int* prev, int i) {
    int j = i, size = 1;
    while (next[j] >= 0 && next[j] != i && size < 5) { j = next[j]; ++size; }
    if (size >= 5) return 0;
    if (next[j] == i) return 1; /* a loop of fewer than five points */
    j = i;
    while (prev[j] >= 0 && size < 5) { j = prev[j]; ++size; }
    return size < 5;
}

static void predecessors(const int* next, const int* alive, int total, int* prev) {
    for (int k = 0; k < total; ++k) prev[k] = -1;
    for (int k = 0; k < total; ++k)
        if (alive[k] && next[k] >= 0) prev[next[k]] = k;
}

/* Keep the alive points in ascending index order and renumber next/prev. */
static void compact(vlbref_channel* ch, int total, const double* pos, const int* next, const int* alive) {
    int* idx = (int*)malloc(sizeof(int) * (size_t)(total > 0 ? total : 1));
    int m = 0;
    for (int k = 0; k < total; ++k) idx[k] = alive[k] ? m++ : -1;
    for (int k = 0; k < total; ++k) {
        if (!alive[k]) continue;
        int nk = idx[k];
        for (int a = 0; a < 3; ++a) ch->pos[3 * nk + a] = pos[3 * k + a];
        ch->next[nk] = next[k] >= 0 ? idx[next[k]] : -1;
    }
    ch->N = m;
    for (int k = 0; k < m; ++k) ch->prev[k] = -1;
    for (int k = 0; k < m; ++k)
        if (ch->next[k] >= 0) ch->prev[ch->next[k]] = k;
    free(idx);
}

/* Remeshing (Sec. II.A, segment lengths kept within [dxi_min, dxi_max]):
 * all decisions are taken on the state before the pass.
 *  split: segment i->q with l > dxi_max gets the arc midpoint
 *         m = s_i + b/2 - (l^2/16)(s''_i + s''_q), appended in ascending i;
 *  merge: point i with both neighbours is a candidate if min(l-, l+) < dxi_min,
 *         |s_q - s_p| <= dxi_max and neither adjacent segment splits; a
 *         candidate is removed unless a neighbouring candidate outranks it
 *         (fmix32 priority, see outranks()); open ends are never removed;
 *  loops and open lines left with fewer than five points are deleted. */
static void remesh(vlbref_channel* ch) {
    const int N = ch->N;
    if (N == 0) return;
    const double dmin = ch->p.dxi_min, dmax = ch->p.dxi_max;
    double* l = (double*)malloc(sizeof(double) * (size_t)N);
    double* spp = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    int* split = (int*)calloc((size_t)N, sizeof(int));
    int* cand = (int*)calloc((size_t)N, sizeof(int));
    int* rem = (int*)calloc((size_t)N, sizeof(int));
    int* rank = (int*)malloc(sizeof(int) * (size_t)N);
    for (int i = 0; i < N; ++i) {
        double sp[3], dxi, lia[3];
        point_geometry(ch, ch->pos, i, sp, &spp[3 * i], &dxi, lia, &l[i]);
        if (ch->next[i] < 0) l[i] = 0.0; /* no segment leaves an end */
    }
    int S = 0;
    for (int i = 0; i < N; ++i) {
        split[i] = ch->next[i] >= 0 && l[i] > dmax;
        rank[i] = split[i] ? S++ : -1;
    }
    for (int i = 0; i < N; ++i) {
        int p = ch->prev[i], q = ch->next[i];
        if (p < 0 || q < 0) continue;
        double pq[3];
        diff3(ch, &ch->pos[3 * q], &ch->pos[3 * p], pq);
        double lmin = l[p] < l[i] ? l[p] : l[i];
        cand[i] = (lmin < dmin) && (norm3(pq) <= dmax) && !split[p] && !split[i];
    }
    for (int i = 0; i < N; ++i) {
        int p = ch->prev[i], q = ch->next[i];
        rem[i] = cand[i] && !(cand[p] && outranks(p, i)) && !(cand[q] && outranks(q, i));
    }
    int total = N + S;
    if (total > ch->cap) { ch->status |= ST_CAPACITY; total = N; S = 0; }
    double* npos = (double*)malloc(sizeof(double) * 3 * (size_t)total);
    int* nnext = (int*)malloc(sizeof(int) * (size_t)total);
    int* alive = (int*)calloc((size_t)total, sizeof(int));
    memcpy(npos, ch->pos, sizeof(double) * 3 * (size_t)N);
    long merges = 0;
    for (int i = 0; i < N; ++i) {
        alive[i] = !rem[i];
        if (rem[i]) { ++merges; continue; }
        int q = ch->next[i];
        if (q < 0) {
            nnext[i] = -1;
        } else if (split[i] && S > 0) {
            int m = N + rank[i];
            double b[3];
            diff3(ch, &ch->pos[3 * q], &ch->pos[3 * i], b);
            for (int a = 0; a < 3; ++a)
                npos[3 * m + a] = ch->pos[3 * i + a] + 0.5 * b[a] - (l[i] * l[i] / 16.0) * (spp[3 * i + a] + spp[3 * q + a]);
            wrap_or_clamp(ch, &npos[3 * m]);
            nnext[i] = m;
            nnext[m] = q;
            alive[m] = 1;
        } else if (rem[q]) {
            nnext[i] = ch->next[q];
        } else {
            nnext[i] = q;
        }
    }
    long small = 0;
    int* alive2 = (int*)malloc(sizeof(int) * (size_t)total);
    int* nprev = (int*)malloc(sizeof(int) * (size_t)total);
    predecessors(nnext, alive, total, nprev);
    for (int k = 0; k < total; ++k) {
        alive2[k] = alive[k] && !in_small_component(nnext, nprev, k);
        if (alive[k] && !alive2[k]) ++small;
    }
    free(nprev);
    ch->n_split += S;
    ch->n_merge += merges;
    ch->n_small += small;
    compact(ch, total, npos, nnext, alive2);
    free(l); free(spp); free(split); free(cand); free(rem); free(rank);
    free(npos); free(nnext); free(alive); free(alive2);
}

/* Reconnection (Sec. II.A: legs exchanged when two vortices come within the
 * resolution; Sec. III.B: within dxi_max).  An exchange acts on two segments
 * a->qa and b->qb and replaces them by a->qb and b->qa.
 *  1. nearest j of each i with |s_j - s_i| < dxi_max, j not within two links of i
 *     (ties to the smaller j);
 *  2. for every mutual nearest pair (i < j) the segment pairs (a, b) in
 *     {(i, j), (i, p(j)), (p(i), j), (p(i), p(j))} are tried in that order and
 *     the first one with the largest length decrease
 *     l_a + l_b - |s_qb - s_a| - |s_qa - s_b| is kept if that decrease is > 0;
 *     (a pair whose a or b is missing or is a line's last point is not tried);
 *  3. exchanges are applied in ascending (d_ij^2, i); one that touches a point
 *     already used by an applied exchange (a, qa, b, qb) is skipped;
 *  4. wall contact: a point with both neighbours that touches a wall's clamp
 *     bound, taken in ascending index and skipped if it or a neighbour is
 *     already used, cuts its line there: it is deleted, its neighbours become
 *     the ends of the cut line and are moved onto the same bound (pinned);
 *  5. loops and open lines left with fewer than five points are deleted. */
static double seg_len(const vlbref_channel* ch, int a, int b) {
    double d[3];
    diff3(ch, &ch->pos[3 * b], &ch->pos[3 * a], d);
    return norm3(d);
}

static void reconnect(vlbref_channel* ch) {
    const int N = ch->N;
    if (N == 0) return;
    const double dmax2 = ch->p.dxi_max * ch->p.dxi_max;
    int* nn = (int*)malloc(sizeof(int) * (size_t)N);
    double* nd2 = (double*)malloc(sizeof(double) * (size_t)N);
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < N; ++i) {
        int p = ch->prev[i], q = ch->next[i];
        int pp = p >= 0 ? ch->prev[p] : -1, qq = q >= 0 ? ch->next[q] : -1;
        int best = -1;
        double bd = 0.0;
        for (int j = 0; j < N; ++j) {
            if (j == i || j == p || j == q || j == pp || j == qq) continue;
            double d[3];
            diff3(ch, &ch->pos[3 * j], &ch->pos[3 * i], d);
            double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(d2 < dmax2)) continue;
            if (best < 0 || d2 < bd) { best = j; bd = d2; }
        }
        nn[i] = best;
        nd2[i] = bd;
    }
    /* candidate exchanges, one per mutual pair, indexed by the pair's i */
    int npairs = 0;
    int* pa = (int*)malloc(sizeof(int) * (size_t)N);
    int* ea = (int*)malloc(sizeof(int) * (size_t)N);
    int* eb = (int*)malloc(sizeof(int) * (size_t)N);
    for (int i = 0; i < N; ++i) {
        int j = nn[i];
        if (j <= i || nn[j] != i) continue;
        int as[4] = {i, i, ch->prev[i], ch->prev[i]};
        int bs[4] = {j, ch->prev[j], j, ch->prev[j]};
        double best = 0.0;
        int pick = -1;
        for (int k = 0; k < 4; ++k) {
            int a = as[k], b = bs[k];
            if (a < 0 || b < 0 || ch->next[a] < 0 || ch->next[b] < 0) continue;
            int qa = ch->next[a], qb = ch->next[b];
            double gain = (seg_len(ch, a, qa) + seg_len(ch, b, qb)) - (seg_len(ch, a, qb) + seg_len(ch, b, qa));
            if (gain > 0.0 && (pick < 0 || gain > best)) { best = gain; pick = k; }
        }
        if (pick < 0) continue;
        ea[i] = as[pick];
        eb[i] = bs[pick];
        pa[npairs++] = i;
    }
    /* order by (d^2, i): insertion sort, the lists are short */
    for (int a = 1; a < npairs; ++a) {
        int key = pa[a], b = a - 1;
        while (b >= 0 && (nd2[pa[b]] > nd2[key] || (nd2[pa[b]] == nd2[key] && pa[b] > key))) {
            pa[b + 1] = pa[b];
            --b;
        }
        pa[b + 1] = key;
    }
    char* claimed = (char*)calloc((size_t)N, 1);
    long applied = 0;
    for (int k = 0; k < npairs; ++k) {
        int i = pa[k];
        int a = ea[i], b = eb[i], qa = ch->next[a], qb = ch->next[b];
        if (claimed[a] || claimed[qa] || claimed[b] || claimed[qb]) continue;
        claimed[a] = claimed[qa] = claimed[b] = claimed[qb] = 1;
        ch->next[a] = qb; ch->prev[qb] = a;
        ch->next[b] = qa; ch->prev[qa] = b;
        ++applied;
    }
    ch->n_reconnect += applied;
    int* alive = (int*)malloc(sizeof(int) * (size_t)N);
    for (int k = 0; k < N; ++k) alive[k] = 1;
    long cuts = 0;
    for (int i = 0; i < N; ++i) {
        int p = ch->prev[i], q = ch->next[i];
        if (p < 0 || q < 0 || claimed[i] || claimed[p] || claimed[q]) continue;
        int code = touching_wall(ch, &ch->pos[3 * i]);
        if (code < 0) continue;
        int ax = code >> 1;
        double bound = (code & 1) ? wall_hi(ch, ax) : wall_lo(ch);
        claimed[i] = claimed[p] = claimed[q] = 1;
        alive[i] = 0;
        ch->next[p] = -1;
        ch->prev[q] = -1;
        ch->pos[3 * p + ax] = bound;
        ch->pos[3 * q + ax] = bound;
        ++cuts;
    }
    ch->n_wallcut += cuts;
    long small = 0;
    for (int k = 0; k < N; ++k) {
        if (!alive[k]) continue;
        alive[k] = !in_small_component(ch->next, ch->prev, k);
        if (!alive[k]) ++small;
    }
    ch->n_small += small;
    if (small > 0 || cuts > 0) {
        double* cpos = (double*)malloc(sizeof(double) * 3 * (size_t)N);
        int* cnext = (int*)malloc(sizeof(int) * (size_t)N);
        memcpy(cpos, ch->pos, sizeof(double) * 3 * (size_t)N);
        memcpy(cnext, ch->next, sizeof(int) * (size_t)N);
        compact(ch, N, cpos, cnext, alive);
        free(cpos); free(cnext);
    }
    free(nn); free(nd2); free(pa); free(ea); free(eb); free(claimed); free(alive);
}

/* ------------------------------------------------------------------- API */

int vlbref_create(const vlbref_params* p, vlbref_channel** out) {
    if (!p || !out) return VLBREF_ERR_INVALID_ARG;
    *out = NULL;
    for (int a = 0; a < 3; ++a)
        if (p->n[a] < 1) return VLBREF_ERR_INVALID_ARG;
    if (!(p->tau > 0.5) || p->stream_axis < 0 || p->stream_axis > 2 || p->max_points < 0 ||
        !(p->rho0 > 0.0) || !(p->rho_s_over_rho_n > 0.0) || !(p->dxi_min > 0.0) || !(p->dxi_max > p->dxi_min))
        return VLBREF_ERR_INVALID_ARG;
    vlbref_channel* ch = (vlbref_channel*)calloc(1, sizeof(vlbref_channel));
    if (!ch) return VLBREF_ERR_OOM;
    ch->p = *p;
    ch->ncell = (long)p->n[0] * p->n[1] * p->n[2];
    const long C = ch->ncell;
    ch->f = (double*)malloc(sizeof(double) * (size_t)(C * Q));
    ch->ftmp = (double*)malloc(sizeof(double) * (size_t)(C * Q));
    ch->RHO = (double*)malloc(sizeof(double) * (size_t)C);
    ch->F = (double*)calloc((size_t)(3 * C), sizeof(double));
    ch->U = (double*)malloc(sizeof(double) * (size_t)(3 * C));
    ch->Vs = (double*)calloc((size_t)p->n[p->stream_axis], sizeof(double));
    ch->cap = p->max_points;
    ch->pos = (double*)calloc((size_t)(3 * (ch->cap + 1)), sizeof(double));
    ch->next = (int*)calloc((size_t)(ch->cap + 1), sizeof(int));
    ch->prev = (int*)calloc((size_t)(ch->cap + 1), sizeof(int));
    ch->vel1 = (double*)calloc((size_t)(3 * (ch->cap + 1)), sizeof(double));
    if (!ch->f || !ch->ftmp || !ch->RHO || !ch->F || !ch->U || !ch->Vs || !ch->pos || !ch->next || !ch->prev || !ch->vel1) {
        vlbref_destroy(ch);
        return VLBREF_ERR_OOM;
    }
    /* initial state: uniform equilibrium at rho0 and init_vn */
    for (int i = 0; i < Q; ++i) {
        double fe = feq_i(i, p->rho0, p->init_vn);
        for (long c = 0; c < C; ++c) ch->f[(long)i * C + c] = fe;
    }
    for (long c = 0; c < C; ++c) ch->RHO[c] = p->rho0;
    for (int a = 0; a < 3; ++a)
        for (long c = 0; c < C; ++c) ch->U[(long)a * C + c] = p->init_vn[a];
    const int ns = p->n[p->stream_axis];
    for (int k = 0; k < ns; ++k) ch->Vs[k] = -(1.0 / p->rho_s_over_rho_n) * p->init_vn[p->stream_axis];
    ch->mass = p->rho0 * (double)C;
    *out = ch;
    return VLBREF_OK;
}

void vlbref_destroy(vlbref_channel* ch) {
    if (!ch) return;
    free(ch->f); free(ch->ftmp); free(ch->RHO); free(ch->F); free(ch->U); free(ch->Vs);
    free(ch->pos); free(ch->next); free(ch->prev); free(ch->vel1);
    free(ch);
}

const char* vlbref_last_error(const vlbref_channel* ch) { return ch ? ch->err : "no channel"; }

int vlbref_seed_vortices(vlbref_channel* ch, const double* xyz, const int32_t* next, int32_t n) {
    if (!ch || n < 0 || (n > 0 && (!xyz || !next))) return VLBREF_ERR_INVALID_ARG;
    if (n > ch->cap) { set_err(ch, "more points than max_points"); return VLBREF_ERR_CAPACITY; }
    int* seen = (int*)calloc((size_t)(n > 0 ? n : 1), sizeof(int));
    for (int i = 0; i < n; ++i) {
        if (next[i] < -1 || next[i] >= n || (next[i] >= 0 && seen[next[i]])) {
            free(seen);
            set_err(ch, "next[] must describe closed loops and open lines");
            return VLBREF_ERR_TOPOLOGY;
        }
        if (next[i] >= 0) seen[next[i]] = 1;
        for (int a = 0; a < 3; ++a) {
            double v = xyz[3 * i + a];
            if (v != v) { free(seen); set_err(ch, "NaN position"); return VLBREF_ERR_INVALID_ARG; }
            if (ch->p.wall[a] && (v <= -0.5 || v >= ch->p.n[a] - 0.5)) {
                free(seen);
                set_err(ch, "point outside the walls");
                return VLBREF_ERR_INVALID_ARG;
            }
        }
    }
    for (int i = 0; i < n; ++i)
        if (next[i] < 0 && !seen[i]) {
            free(seen);
            set_err(ch, "isolated point");
            return VLBREF_ERR_TOPOLOGY;
        }
    free(seen);
    /* open ends go onto the nearest wall bound (within dxi_max of it) */
    double* tmp = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    int* tprev = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) tmp[3 * i + a] = xyz[3 * i + a];
        wrap_or_clamp(ch, &tmp[3 * i]);
        tprev[i] = -1;
    }
    for (int i = 0; i < n; ++i)
        if (next[i] >= 0) tprev[next[i]] = i;
    for (int i = 0; i < n; ++i) {
        if (next[i] >= 0 && tprev[i] >= 0) continue;
        int best_a = -1;
        double best_d = 0.0, best_b = 0.0;
        for (int a = 0; a < 3; ++a) {
            if (!ch->p.wall[a]) continue;
            double lo = wall_lo(ch), hi = wall_hi(ch, a);
            double dl = tmp[3 * i + a] - lo, dh = hi - tmp[3 * i + a];
            if (best_a < 0 || dl < best_d) { best_a = a; best_d = dl; best_b = lo; }
            if (dh < best_d) { best_a = a; best_d = dh; best_b = hi; }
        }
        if (best_a < 0 || best_d > ch->p.dxi_max) {
            free(tmp); free(tprev);
            set_err(ch, "open end farther than dxi_max from every wall");
            return VLBREF_ERR_TOPOLOGY;
        }
        tmp[3 * i + best_a] = best_b;
    }
    ch->N = n;
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) ch->pos[3 * i + a] = tmp[3 * i + a];
        ch->next[i] = next[i];
        ch->prev[i] = tprev[i];
    }
    free(tmp); free(tprev);
    return VLBREF_OK;
}

int vlbref_run_phases(vlbref_channel* ch, int32_t mask) {
    if (!ch) return VLBREF_ERR_INVALID_ARG;
    if (mask & VLBREF_PHASE_LBM) lbm_pass(ch);
    if (mask & VLBREF_PHASE_VFM) vfm_advance(ch);
    if (mask & VLBREF_PHASE_REMESH) remesh(ch);
    if (mask & VLBREF_PHASE_RECONNECT) reconnect(ch);
    if (ch->status & ST_NAN) { set_err(ch, "NaN in the lattice"); return VLBREF_ERR_NAN; }
    if (ch->status & ST_CAPACITY) { set_err(ch, "point capacity exceeded"); return VLBREF_ERR_CAPACITY; }
    if (ch->status & ST_MACH) { set_err(ch, "Mach number >= 0.05"); return VLBREF_ERR_MACH; }
    return VLBREF_OK;
}

int vlbref_step(vlbref_channel* ch, int32_t nsteps) {
    if (!ch || nsteps < 0) return VLBREF_ERR_INVALID_ARG;
    for (int s = 0; s < nsteps; ++s) {
        int rc = vlbref_run_phases(ch, VLBREF_PHASE_ALL);
        ch->steps++;
        if (rc) return rc;
    }
    return VLBREF_OK;
}

static double line_length(const vlbref_channel* ch) {
    double L = 0.0;
    for (int i = 0; i < ch->N; ++i) {
        if (ch->next[i] < 0) continue;
        double b[3];
        diff3(ch, &ch->pos[3 * ch->next[i]], &ch->pos[3 * i], b);
        L += norm3(b);
    }
    return L;
}

/* Line length per stream plane (the profile behind the line density L(x) of
 * Sec. IV, Fig. 8b): each segment's length goes to the plane nearest its
 * midpoint (periodic axes wrap, walls clamp). */
static void line_profile(const vlbref_channel* ch, double* prof) {
    const int sa = ch->p.stream_axis, ns = ch->p.n[sa];
    for (int k = 0; k < ns; ++k) prof[k] = 0.0;
    for (int i = 0; i < ch->N; ++i) {
        if (ch->next[i] < 0) continue;
        double b[3];
        diff3(ch, &ch->pos[3 * ch->next[i]], &ch->pos[3 * i], b);
        double mid = ch->pos[3 * i + sa] + 0.5 * b[sa];
        int k = (int)floor(mid + 0.5);
        if (!ch->p.wall[sa]) k = ((k % ns) + ns) % ns;
        else k = k < 0 ? 0 : (k > ns - 1 ? ns - 1 : k);
        prof[k] += norm3(b);
    }
}

int vlbref_line_length(vlbref_channel* ch, double* out) {
    if (!ch || !out) return VLBREF_ERR_INVALID_ARG;
    *out = line_length(ch);
    return VLBREF_OK;
}

int vlbref_read_fields(vlbref_channel* ch, int32_t which, void* dst, size_t bytes, size_t* written) {
    if (!ch || !dst) return VLBREF_ERR_INVALID_ARG;
    const long C = ch->ncell;
    size_t need = 0;
    switch (which) {
    case VLBREF_FIELD_RHO: need = sizeof(double) * (size_t)C; break;
    case VLBREF_FIELD_U: case VLBREF_FIELD_FORCE: case VLBREF_FIELD_ULAST: need = sizeof(double) * 3 * (size_t)C; break;
    case VLBREF_FIELD_FSTAR: need = sizeof(double) * Q * (size_t)C; break;
    case VLBREF_FIELD_POS: case VLBREF_FIELD_VEL: need = sizeof(double) * 3 * (size_t)ch->N; break;
    case VLBREF_FIELD_NEXT: need = sizeof(int32_t) * (size_t)ch->N; break;
    case VLBREF_FIELD_PLANE_VS: case VLBREF_FIELD_LINE_PROFILE:
        need = sizeof(double) * (size_t)ch->p.n[ch->p.stream_axis];
        break;
    case VLBREF_FIELD_STATS: need = sizeof(double) * 16; break;
    default: return VLBREF_ERR_INVALID_ARG;
    }
    if (bytes < need) { set_err(ch, "destination too small"); return VLBREF_ERR_INVALID_ARG; }
    double* d = (double*)dst;
    if (which == VLBREF_FIELD_RHO || which == VLBREF_FIELD_U) {
        for (int z = 0; z < ch->p.n[2]; ++z)
            for (int y = 0; y < ch->p.n[1]; ++y)
                for (int x = 0; x < ch->p.n[0]; ++x) {
                    long c = cell_index(ch, x, y, z);
                    double fin[Q], rho, u[3], Ft[3];
                    for (int i = 0; i < Q; ++i) fin[i] = pulled(ch, ch->f, i, x, y, z);
                    moments(ch, fin, c, &rho, u, Ft);
                    if (which == VLBREF_FIELD_RHO) d[c] = rho;
                    else for (int a = 0; a < 3; ++a) d[(long)a * C + c] = u[a];
                }
    } else if (which == VLBREF_FIELD_FSTAR) {
        memcpy(d, ch->f, need);
    } else if (which == VLBREF_FIELD_FORCE) {
        memcpy(d, ch->F, need);
    } else if (which == VLBREF_FIELD_ULAST) {
        memcpy(d, ch->U, need);
    } else if (which == VLBREF_FIELD_POS) {
        memcpy(d, ch->pos, need);
    } else if (which == VLBREF_FIELD_VEL) {
        memcpy(d, ch->vel1, need);
    } else if (which == VLBREF_FIELD_NEXT) {
        memcpy(dst, ch->next, need);
    } else if (which == VLBREF_FIELD_PLANE_VS) {
        memcpy(d, ch->Vs, need);
    } else if (which == VLBREF_FIELD_LINE_PROFILE) {
        line_profile(ch, d);
    } else {
        for (int k = 0; k < 16; ++k) d[k] = 0.0;
        d[0] = ch->N; d[1] = ch->status; d[2] = ch->mass; d[3] = line_length(ch);
        d[4] = ch->max_mach; d[5] = (double)ch->n_split; d[6] = (double)ch->n_merge;
        d[7] = (double)ch->n_reconnect; d[8] = (double)ch->n_small; d[9] = (double)ch->steps;
        d[10] = ch->mom[0]; d[11] = ch->mom[1]; d[12] = ch->mom[2];
        d[13] = (double)ch->n_wallcut;
    }
    if (written) *written = need;
    return VLBREF_OK;
}

int vlbref_write_fields(vlbref_channel* ch, int32_t which, const void* src, size_t bytes) {
    if (!ch || !src) return VLBREF_ERR_INVALID_ARG;
    const long C = ch->ncell;
    if (which == VLBREF_FIELD_FSTAR) {
        if (bytes != sizeof(double) * Q * (size_t)C) return VLBREF_ERR_INVALID_ARG;
        memcpy(ch->f, src, bytes);
    } else if (which == VLBREF_FIELD_FORCE) {
        if (bytes != sizeof(double) * 3 * (size_t)C) return VLBREF_ERR_INVALID_ARG;
        memcpy(ch->F, src, bytes);
    } else if (which == VLBREF_FIELD_ULAST) {
        if (bytes != sizeof(double) * 3 * (size_t)C) return VLBREF_ERR_INVALID_ARG;
        memcpy(ch->U, src, bytes);
    } else if (which == VLBREF_FIELD_PLANE_VS) {
        if (bytes != sizeof(double) * (size_t)ch->p.n[ch->p.stream_axis]) return VLBREF_ERR_INVALID_ARG;
        memcpy(ch->Vs, src, bytes);
    } else {
        return VLBREF_ERR_INVALID_ARG;
    }
    return VLBREF_OK;
}

/* --------------------------------------------------------- component calls */

void vlbref_lattice(int32_t* c, double* w, int32_t* opp) {
    for (int i = 0; i < Q; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = CV[i][a];
        w[i] = WV[i];
        opp[i] = opposite(i);
    }
}

void vlbref_feq(double rho, const double* u, double* out) {
    for (int i = 0; i < Q; ++i) out[i] = feq_i(i, rho, u);
}

void vlbref_force_terms(const double* u, const double* F, double tau, double* out) {
    for (int i = 0; i < Q; ++i) out[i] = force_i(i, u, F, tau);
}

void vlbref_segment_velocity(const double* r, const double* s1, const double* s2, double kappa, double* out) {
    double R1[3], d[3];
    for (int k = 0; k < 3; ++k) {
        R1[k] = s1[k] - r[k];
        d[k] = s2[k] - s1[k];
        out[k] = 0.0;
    }
    segment_add(R1, d, kappa, out);
}

int vlbref_geometry(vlbref_channel* ch, double* sp, double* spp, double* dxi, double* lia) {
    if (!ch) return VLBREF_ERR_INVALID_ARG;
    for (int i = 0; i < ch->N; ++i)
        point_geometry(ch, ch->pos, i, &sp[3 * i], &spp[3 * i], &dxi[i], &lia[3 * i], NULL);
    return VLBREF_OK;
}

int vlbref_point_velocity(vlbref_channel* ch, double* vel, double* vbs) {
    if (!ch || !vel) return VLBREF_ERR_INVALID_ARG;
    filament_velocity(ch, ch->pos, vel, vbs, 0);
    return VLBREF_OK;
}

int vlbref_interp(vlbref_channel* ch, const double* xyz, int32_t n, double* out) {
    if (!ch) return VLBREF_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) interp_u(ch, ch->U, &xyz[3 * i], &out[3 * i]);
    return VLBREF_OK;
}

int vlbref_spread(vlbref_channel* ch, const double* xyz, const double* g, int32_t n) {
    if (!ch) return VLBREF_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) spread_g(ch, &xyz[3 * i], &g[3 * i]);
    return VLBREF_OK;
}
