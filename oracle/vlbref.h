/*
 * vlbref.h -- plain FP64 CPU oracle of one coupled vortex-filament /
 * lattice-Boltzmann time step (Inui & Tsubota, arXiv 2108.04435).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists so that the CUDA path can be
 * checked against a slow, obviously correct restatement of the paper's method.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Units: lattice units throughout (dx = dt = 1 for the LBM, Sec. II.B).
 * Lattice nodes sit at integer coordinates 0..n-1; a solid wall on an axis sits
 * half-way outside the first and last node (halfway bounce-back).
 *
 * Population order used for every populations array exported here (Table I,
 * written 0-based):
 *   0 rest; 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z;
 *   7 (+1,+1,0)  8 (-1,-1,0)  9 (+1,-1,0) 10 (-1,+1,0)
 *  11 (+1,0,+1) 12 (-1,0,-1) 13 (+1,0,-1) 14 (-1,0,+1)
 *  15 (0,+1,+1) 16 (0,-1,-1) 17 (0,+1,-1) 18 (0,-1,+1)
 * Field arrays are structure-of-arrays with x fastest: a[c][z][y][x].
 */
#ifndef VLBREF_H
#define VLBREF_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t n[3];            /* cells along x, y, z */
    int32_t wall[3];         /* 0 periodic, 1 halfway bounce-back walls on both faces */
    int32_t stream_axis;     /* counterflow axis (heater faces, V_s planes) */
    int32_t vfm_substeps;    /* RK4 substeps per lattice step (>= 1) */
    int32_t couple;          /* 1: spread the friction reaction onto the lattice (Eq. 10-11) */
    int32_t force_form;      /* 0: f of Eq. 10 as printed; 1: f = rho_s kappa (Eq. 10 rhs) x s' (Magnus drag) */
    int32_t max_points;      /* filament point capacity */
    int32_t reserved;
    int32_t wall_images;     /* 1: v_s,b from first-order mirror images across each solid wall face (Sec. II.A) */
    int32_t reserved2;
    double tau, rho0;        /* BGK relaxation time (> 1/2), reference density */
    double body_force[3];    /* uniform body force added to the force grid */
    double heater_vn;        /* normal velocity injected at the low stream face, removed at the high face */
    double pin_vn;           /* periodic stream axis: plane 0 reset to f^eq(rho, pin_vn e_s); 0 = off */
    double init_vn[3];       /* initial uniform normal-fluid velocity */
    double kappa, alpha, alpha_p, rho_s_over_rho_n, core_a;
    double dxi_min, dxi_max;
} vlbref_params;

typedef struct vlbref_channel vlbref_channel;

enum {
    VLBREF_OK = 0,
    VLBREF_ERR_INVALID_ARG = -1,
    VLBREF_ERR_OOM = -2,
    VLBREF_ERR_CAPACITY = -3,
    VLBREF_ERR_TOPOLOGY = -4,
    VLBREF_ERR_MACH = -5,
    VLBREF_ERR_NAN = -6
};

enum { VLBREF_PHASE_LBM = 1, VLBREF_PHASE_VFM = 2, VLBREF_PHASE_REMESH = 4,
       VLBREF_PHASE_RECONNECT = 8, VLBREF_PHASE_ALL = 15 };

enum {
    VLBREF_FIELD_RHO = 0,      /* [C]      density of the streamed populations (next step's moments) */
    VLBREF_FIELD_U = 1,        /* [3][C]   half-force shifted velocity of the same */
    VLBREF_FIELD_FSTAR = 2,    /* [19][C]  post-collision populations */
    VLBREF_FIELD_FORCE = 3,    /* [3][C]   force grid */
    VLBREF_FIELD_POS = 4,      /* [N][3]   filament points */
    VLBREF_FIELD_NEXT = 5,     /* [N]      int32 successor index, -1 at the last point of an open line */
    VLBREF_FIELD_PLANE_VS = 6, /* [n_s]    superfluid velocity per stream plane (Eq. 18) */
    VLBREF_FIELD_STATS = 7,    /* [16]     see vlbref.c */
    VLBREF_FIELD_VEL = 8,      /* [N][3]   stage-1 ds/dt of the last filament advance */
    VLBREF_FIELD_ULAST = 9,    /* [3][C]   velocity u^n seen by the last filament advance */
    VLBREF_FIELD_LINE_PROFILE = 10 /* [n_s] line length per stream plane */
};

int  vlbref_create(const vlbref_params* p, vlbref_channel** out);
void vlbref_destroy(vlbref_channel* ch);
const char* vlbref_last_error(const vlbref_channel* ch);
/* next[i] = successor of point i, or -1 where an open line ends.  Closed loops
 * and open lines only (no point has two predecessors; no isolated point).  An
 * open end must lie within dxi_max of a wall's clamp bound and is moved onto
 * the nearest one: it is pinned to that wall. */
int  vlbref_seed_vortices(vlbref_channel* ch, const double* xyz, const int32_t* next, int32_t n);
int  vlbref_step(vlbref_channel* ch, int32_t nsteps);
int  vlbref_run_phases(vlbref_channel* ch, int32_t phase_mask);
int  vlbref_read_fields(vlbref_channel* ch, int32_t which, void* dst, size_t bytes, size_t* written);
int  vlbref_write_fields(vlbref_channel* ch, int32_t which, const void* src, size_t bytes);
int  vlbref_line_length(vlbref_channel* ch, double* out);

/* component entry points used by the pin tests */
void vlbref_lattice(int32_t* c /*[19][3]*/, double* w /*[19]*/, int32_t* opp /*[19]*/);
void vlbref_feq(double rho, const double* u /*[3]*/, double* out /*[19]*/);
void vlbref_force_terms(const double* u, const double* F, double tau, double* out /*[19]*/);
void vlbref_segment_velocity(const double* r, const double* s1, const double* s2, double kappa, double* out);
int  vlbref_geometry(vlbref_channel* ch, double* sp, double* spp, double* dxi, double* lia);
int  vlbref_point_velocity(vlbref_channel* ch, double* vel, double* vbs);
int  vlbref_interp(vlbref_channel* ch, const double* xyz, int32_t n, double* out);
int  vlbref_spread(vlbref_channel* ch, const double* xyz, const double* g, int32_t n);

#ifdef __cplusplus
}
#endif
#endif
