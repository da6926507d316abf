/*
 * CPU FP64 oracle for the third-order gas-kinetic scheme with compact
 * least-squares (CLS) reconstruction on triangles (Li, Zhong & Zhuo,
 * "A third order gas-kinetic scheme for unstructured grid").
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, plain reference that the
 * CUDA library is checked against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Internal header of the oracle (not part of the library's public include/).
 */
#ifndef OR_INTERNAL_H
#define OR_INTERNAL_H

#include <stdint.h>

typedef struct or_params {
    double gamma;       /* ratio of specific heats                               */
    double cfl;         /* CFL number of the explicit step                       */
    double mu;          /* dynamic viscosity; 0 selects the inviscid tau, Eq. (39) */
    double cls_w;       /* derivative weight w of Eq. (29)                       */
    int    gmres_m;     /* restart length                                        */
    int    gmres_maxit; /* iteration cap per variable                            */
    double gmres_rtol;  /* relative residual target                              */
    int    tau2_exact;  /* 1: c4..c6 with the 2 tau^2 (1 - e^{-t/tau}) term       */
    int    slope0_mode; /* interface-equilibrium derivatives: 0 mean of L/R,      */
                        /* 1 kinetic weighting (half-space moments of L/R slopes) */
    int    limiter;     /* 1: shock detector + DWBAP limiter (Sec. III.C); 2: the
                           detector with first order in limited cells (robust)   */
    int    second_order; /* 1: k_i = 1 for every cell (linear CLS reconstruction) */
    double prandtl;     /* Prandtl number of the heat-flux correction (1: none)  */
    int    limit_char;  /* 1: DWBAP in characteristic variables (Sec. IV.B)       */
    int    cls_global;  /* 1: the global normal equations C^T C u = C^T b of the
                           whole mesh (Eq. (33), symmetric positive definite)
                           instead of each cell's own least-squares equations    */
    int    cls_M;       /* highest derivative order p <= M <= k of the CLS
                           equations of Eq. (29) (default 1; 0 needs k = 1)      */
} or_params;

/* Boundary tags (same numbering as the input generator). */
enum { OR_INTERIOR = 0, OR_PERIODIC = 1, OR_DIRICHLET = 2, OR_OUTFLOW = 3,
       OR_SLIP = 4, OR_NOSLIP = 5 };

typedef struct or_csr {
    int n, nnz;
    int *rowptr, *col;
    double *val;
} or_csr;

typedef struct or_mesh {
    or_params prm;
    int64_t n_nodes, n_tri, n_face;
    double *nodes;          /* 2*n_nodes                                       */
    int *tri;               /* 3*n_tri, counter-clockwise                      */
    int *face;              /* 5*n_face: n0 n1 l r tag                          */
    double *shift;          /* 2*n_face                                        */
    double *bc;             /* 4*n_face                                        */
    /* cell geometry */
    double *area, *cx, *cy, *crad, *h, *inrad, *mxx, *mxy, *myy;
    int *korder;            /* k_i of Eq. (28)                                 */
    int *cface;             /* 3 faces per cell (-1 unused)                     */
    /* face geometry */
    double *fnx, *fny, *flen, *gx, *gy;   /* gx, gy: 2 Gauss points per face */
    /* CLS system */
    int *dof_off;           /* offset of cell i's unknowns; n_i = 5 or 2       */
    int ndof;
    int *nb_cnt;            /* neighbours per cell (<= 3)                      */
    int *nb_cell;           /* 3 per cell                                      */
    double *nb_dx, *nb_dy;  /* offset added to the neighbour's coordinates     */
    double *a0;             /* 3*5 per cell: weighted row 0 of A_ij (RHS rows) */
    or_csr K;               /* per-cell normal equations, natural order        */
    int *perm;              /* RCM: new -> old cell                            */
    int *dperm, *dinv;      /* dof permutation new -> old, old -> new          */
    or_csr Kp;              /* permuted matrix                                  */
    or_csr LU;              /* scalar ILU(0) of Kp                              */
    int *diag_pos;          /* position of the diagonal in LU rows              */
    double *warm;           /* 4*ndof previous solution (natural dof order)    */
} or_mesh;

/* geometry and CLS (or_geom_cls.c) */
int  or_build_geometry(or_mesh *m);
int  or_build_cls(or_mesh *m);
int  or_build_rcm(or_mesh *m);
void or_cls_rhs_var(const or_mesh *m, const double *ubar, double *rhs);

/* linear algebra (or_linsolve.c) */
void or_csr_free(or_csr *a);
void or_csr_matvec(const or_csr *a, const double *x, double *y);
int  or_ilu0(const or_csr *a, or_csr *lu, int **diag_pos);
void or_ilu0_apply(const or_csr *lu, const int *diag_pos, const double *r, double *z);
int  or_gmres(const or_csr *a, const or_csr *lu, const int *diag_pos, const double *b,
              double *x, int m, int maxit, double rtol, int *iters, double *relres);
int  or_dense_lu_solve(int n, double *a, double *b);

/* kinetic part (or_kinetic.c) */
void or_gauss_legendre(int n, double *x, double *w);
void or_time_integrals(double dt, double tau, int tau2_exact, double *c);
int  or_interface_w0(const double *wl, const double *wr, double gamma, int mode, double *w0);
int  or_gp_flux(const double *wl, const double *wr, double dt, const or_params *prm,
                double *f, double *aux);

/* boundary ghost states (or_scheme.c) */
void or_ghost_rows(int tag, const double *bc, double nx, double ny, double gamma, const double *wl, double *wr);

/* limiter (or_limiter.c) */
int  or_limit(const or_mesh *m, const double *w, const double *coef, double *coef_out, int32_t *flag);
void or_char_basis(const double *W, double gamma, double nx, double ny, double *R, double *L);

#endif
