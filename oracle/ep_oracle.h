/*
 * ep_oracle.h -- interface of the plain FP64 CPU oracle (test infrastructure
 * only; see ep_oracle.c for the definitions and their sources in the thesis).
 */
#ifndef EP_ORACLE_H
#define EP_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OG_MONO 0
#define OG_BI 1

typedef struct {
    int nx, ny, nz;
    double dx;                  /* mm */
    const unsigned char *mask;  /* n, 1 = tissue */
    const double *fib;          /* 3n, (fx, fy, fz) per voxel; unit or zero */
    const unsigned char *torso; /* NULL, or n: 1 = conducting torso (bath) voxel outside the tissue */
    double sig_o;               /* isotropic torso conductivity (mS/mm) */
} og_grid;

typedef struct {
    double tau_in, tau_out, tau_open, tau_close, v_gate;
    double sig_iL, sig_iT, sig_eL, sig_eT;
    double lam, K, dt, omega, rel_tol;
    int check_every, max_iter, model;
    int diffusion;              /* OG_EXPLICIT or OG_IMPLICIT (Eq. iejac1) */
    int solver;                 /* elliptic solve: OG_JACOBI (Eq. dampjac1), OG_CHEBYSHEV or OG_GAUSS_SEIDEL */
    double cheb_lmin, cheb_lmax;   /* spectral interval of D^-1 A for OG_CHEBYSHEV */
    double sig_o;               /* torso conductivity, used once og_set_torso is called */
} og_params;

#define OG_JACOBI 0
#define OG_CHEBYSHEV 1
#define OG_GAUSS_SEIDEL 2

#define OG_EXPLICIT 0
#define OG_IMPLICIT 1

typedef struct {
    int lo[3], hi[3];           /* voxel box [lo, hi) */
    double t_start, dur, amp;   /* ms, ms, 1/ms */
} og_stim;

typedef struct og_sim og_sim;

void og_apply_L(const og_grid *g, double sL, double sT, const double *u, double *out);
void og_diag_L(const og_grid *g, double sL, double sT, double *diag);
int og_components(const og_grid *g, int *comp);
double og_default_omega(double sL, double sT);
int og_jacobi(const og_grid *g, double sL, double sT, const double *b, double *x,
              double omega, double tol, int m, int max_iter, int *iters, double *relres);
int og_ie_jacobi(const og_grid *g, double sL, double sT, double alpha, const double *f, double *x,
                 double tol, int m, int max_iter, int *iters, double *relres);
int og_chebyshev(const og_grid *g, double sL, double sT, const double *b, double *x, double lmin, double lmax,
                 double tol, int m, int max_iter, int *iters, double *relres);
int og_gauss_seidel(const og_grid *g, double sL, double sT, const double *b, double *x, double omega,
                    double tol, int m, int max_iter, int *iters, double *relres);

og_sim *og_create(int nx, int ny, int nz, double dx, const unsigned char *mask,
                  const double *fib, const og_params *p, const og_stim *stim, int nstim);
void og_destroy(og_sim *s);
int og_set_torso(og_sim *s, const unsigned char *torso);
void og_set_state(og_sim *s, const double *v, const double *w, const double *ve, long step);
void og_get_state(const og_sim *s, double *v, double *w, double *ve, double *tact, long *step);
int og_step(og_sim *s, int *iters, double *relres);
int og_run(og_sim *s, int nsteps, int *last_iters, double *last_relres);
int og_ncomp(const og_sim *s);
long og_total_iters(const og_sim *s);
long og_ie_total_iters(const og_sim *s);
int og_num_threads(void);

/* Geometry by signed distance functions (Sec. "Geometry"): a postfix program
 * of nodes.  Primitives push their value at the point, operators pop their
 * operands and push the result. */
#define OG_SDF_CUBOID 0          /* a, b, c: half-extents */
#define OG_SDF_ELLIPSOID 1       /* a, b, c: semi-axes */
#define OG_SDF_CYLINDER 2        /* a: radius, b: half-height (axis z) */
#define OG_SDF_CONE 3            /* a: radius at z = 0, b: half-height, c: radius slope (axis z) */
#define OG_SDF_UNION 10
#define OG_SDF_INTERSECT 11
#define OG_SDF_SUBTRACT 12       /* first minus second */
#define OG_SDF_HOLLOW 13         /* |s| - a */
#define OG_SDF_SMOOTH_UNION 14   /* smoothed minimum with width a */

typedef struct {
    int op;
    float a, b, c;
    float centre[3];             /* mm, scene frame */
    float rot[9];                /* row-major: local = rot (x - centre) */
} og_sdf_node;

#define OG_REGION_MYOCARDIUM 1   /* tissue, helical fibres */
#define OG_REGION_FAST 2         /* tissue, fibre = scale * axis */
#define OG_REGION_INSULATOR 3    /* not tissue (zero conductivity) */

typedef struct {
    int first, count, kind;      /* its program: nodes [first, first + count) */
    float axis[3];
    float scale;
} og_sdf_region;

float og_sdf_eval(const og_sdf_node *nodes, int count, const float x[3]);
int og_sdf_encode(const og_sdf_node *nodes, const og_sdf_region *regions, int n_regions, int nx, int ny, int nz,
                  float dx, const float origin[3], double helix_rad, unsigned char *label, unsigned char *mask,
                  double *fib, unsigned char *vclass);

#ifdef __cplusplus
}
#endif
#endif
