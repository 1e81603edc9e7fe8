/*
 * gals_oracle.h -- plain FP64 reference implementation of the gradient-augmented
 * level set (GALS) step of Nave, Rosales and Seibold (arXiv 0905.3409).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA path.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no source, header, table or helper with the CUDA library, and it never
 * loads that library.  Everything here is deliberately slow and direct: no blocking,
 * no sum factorisation, no fusion.  Each function cites the passage of the paper it
 * follows.
 *
 * Conventions used throughout the oracle:
 *   - dim p in {1,2,3}; nodes per axis n[i] >= 2 (>= 4 for the cross stencils);
 *     node coordinate x_i = lo[i] + idx_i * h[i]; x is the fastest-varying index.
 *   - Dv[3*i+j] = d v_i / d x_j  (the usual Jacobian; the paper's grad v is its
 *     transpose, Sec. 4).  J[3*i+j] = d foot_i / d x_j, so the paper's grad(foot)
 *     is J^T and the gradient update is psi+ = J^T grad H (eq. superconsistency).
 *   - Planes: 1D [phi, phi_x]; 2D [phi, phi_x, phi_y, phi_xy];
 *     3D [phi, phi_x, phi_y, phi_z, phi_xy, phi_xz, phi_yz, phi_xyz].
 *   - Hermite cell data are indexed data[v*2^p + a], v, a in {0,1}^p packed as
 *     bit i = component i (Def. "data for phi on C").
 */
#ifndef GALS_ORACLE_H
#define GALS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* velocity kinds (analytic fields with exact Dv, Sec. 4 "exactly accessible") */
enum {
    ORC_VEL_CONST = 0,     /* v = c */
    ORC_VEL_ROTATION = 1,  /* rigid rotation about center, angular speed omega (Sec. 6.2.1) */
    ORC_VEL_VORTEX2D = 2,  /* single vortex, stream fn (1/pi)cos(pi t/T)sin^2(pi x)sin^2(pi y) (Sec. 6.1.2) */
    ORC_VEL_DEFORM3D = 3,  /* LeVeque 3D deformation modulated by cos(pi t/T) (Sec. 6.2.4) */
    ORC_VEL_PSEUDO1D = 4,  /* eq. velocity_1 (Sec. 6.1.1) */
    ORC_VEL_FOURIER2D = 5, /* stream fn sum_m a_m sin(k pi x) sin(l pi y) cos(2 pi n t + chi) */
    ORC_VEL_WAVES2D = 6    /* stream fn sum_m a_m sin(kx x + ky y + phase) cos(2 pi n t + chi)
                              (plane waves of any wave vector; not in the paper) */
};

/* EULER, RK3: superconsistent traces (Sec. 5.1 examples); psi+ = J^T grad H(foot).
 * HEUN_PSI: the CIR form of Sec. 4 with the step-3 choice the paper names for gradients:
 * the foot by the Shu-Osher RK3 trace, psi(foot) = grad H(foot), then
 * d psi / d tau = -grad v . psi (eq. cir_evolution_psi; (grad v)_ij = dv_j/dx_i) integrated
 * forward from (foot, t) to (node, t + dt) by one step of Heun's method (explicit
 * trapezoidal rule). */
enum { ORC_TRACE_EULER = 0, ORC_TRACE_RK3 = 1, ORC_TRACE_HEUN_PSI = 2 };
/* Cross derivatives of the interpolation data (Sec. 2.3):
 * CENTRAL: approach (A), node values rebuilt from the new gradients after every step;
 * ZERO: zero cross planes after the step (tests only);
 * CELL: approach (B), computed per cell from the gradients at the cell's own vertices
 *   (edge-centre differences extrapolated to each vertex with weights 3/4, 3/4, -1/4,
 *   -1/4; in 3D within the vertex's facet of the cell; phi_xyz from the double difference
 *   of psi_z over the vertex's x-y facet).  No node value exists, so the state's cross
 *   planes are zero after a step. */
enum { ORC_CROSS_CENTRAL = 0, ORC_CROSS_ZERO = 1, ORC_CROSS_CELL = 2 };

typedef struct {
    int kind;
    double T;          /* modulation period for VORTEX2D / DEFORM3D */
    double omega;      /* ROTATION angular speed */
    double center[3];  /* ROTATION center */
    double c[3];       /* CONST velocity */
    int nmodes;        /* FOURIER2D, WAVES2D: number of modes */
    const double *modes; /* FOURIER2D: 5 doubles per mode: a, k, l, n, chi;
                            WAVES2D: 6 doubles per mode: a, kx, ky, phase, n, chi */
} orc_velocity;

typedef struct {
    int dim;
    int n[3];
    double lo[3];
    double h[3];
    int cross;         /* cross derivatives the diagnostics' interpolant uses: ORC_CROSS_CENTRAL
                          (the stored planes) or ORC_CROSS_CELL (approach B, per cell) */
} orc_grid;

/* 1-cubic basis (eq. 1-cubic_basis_functions): w[v*2+a](xi) and d/dxi */
void orc_basis1d(double xi, double w[4], double dw[4]);

/* p-cubic Hermite interpolant on one cell (eq. p-cubic_interpolant), direct 4^p-term
 * sum.  data: 4^p scalars; h: cell edge lengths; xi: relative coords in [0,1]^p.
 * Returns H and grad H (physical derivatives, 1/h_i applied). */
void orc_hermite_cell(int dim, const double *data, const double *h,
                      const double *xi, double *H, double *gradH);

/* the same sum with the second derivatives: hessH[j*dim+k] = d^2 H / dx_j dx_k
 * (Sec. 3.4: derivative quantities inside a cell from the interpolant itself) */
void orc_hermite_cell2(int dim, const double *data, const double *h, const double *xi,
                       double *H, double *gradH, double *hessH);

/* velocity and its Jacobian at (x, t) */
void orc_vel_eval(const orc_velocity *vel, int dim, const double *x, double t,
                  double v[3], double Dv[9]);

/* approximate backward characteristic from x at time t+dt to time t, with its
 * Jacobian (Ex. "superconsistent forward Euler" and Ex. "superconsistent Shu-Osher") */
void orc_trace(int scheme, const orc_velocity *vel, int dim, const double *x,
               double t, double dt, double foot[3], double J[9]);

/* classical RK4 with m sub-steps for the backward flow map and its Jacobian
 * (variational equation dJ/dtau = Dv J); a high-accuracy judge for traces */
void orc_flowmap_rk4(const orc_velocity *vel, int dim, const double *x, double t,
                     double dt, int m, double foot[3], double J[9]);

/* cross-derivative reconstruction from the gradient planes (Sec. 2.3, approach A,
 * central differences; one-sided second order at the boundary).  planes as above. */
void orc_recon_cross(const orc_grid *g, double *const *planes);

/* one node of the step: new phi and psi at node (i,j,k) from the old state
 * (steps 1-2 of Sec. 4 with the superconsistent update, eq. superconsistency) */
void orc_node_update(const orc_grid *g, const orc_velocity *vel, int trace, int cross,
                     double t, double dt, const double *const *in,
                     int i, int j, int k, double *phi, double psi[3]);

/* approach (B): replace the cross entries of a cell's gathered data (data[v * 2^p + a],
 * vertex v = vx + 2 vy + 4 vz, derivative multi-index a, bit i = d/dx_i) by the
 * cell-based approximations from the same data's gradient entries */
void orc_cross_cell(int dim, const double *h, double *data);

/* full step t -> t+dt over all nodes, then cross reconstruction (M = P A, Sec. 5.2) */
void orc_step(const orc_grid *g, const orc_velocity *vel, int trace, int cross,
              double t, double dt, const double *const *in, double *const *out,
              int nthreads);

/* full step with the backward map given instead of traced (the learned flow map
 * supplies it): node x_j's foot is x_j + disp[d][j] and its Jacobian
 * J[a][b] = d foot_a / d x_b is jac[dim*a + b][j]; then Sec. 4 step 2 at that foot,
 * psi+ = J^T grad H (eq. superconsistency) and the cross reconstruction, as orc_step */
void orc_step_given(const orc_grid *g, int cross, const double *const *in,
                    const double *const *disp, const double *const *jac, double *const *out,
                    int nthreads);

/* new state (all planes) at a list of nodes only; for parity checks at full size */
void orc_step_nodes(const orc_grid *g, const orc_velocity *vel, int trace, int cross,
                    double t, double dt, const double *const *in, long nsel,
                    const long *sel, double *outv, int nthreads);

/* new state of a band of the outermost axis only: rows [b0,b1) in 2D, z-slices in 3D
 * (the cross stencils never leave a row / slice, so the band is exact); out planes hold
 * the band's nodes contiguously */
void orc_step_band(const orc_grid *g, const orc_velocity *vel, int trace, int cross,
                   double t, double dt, const double *const *in, int b0, int b1,
                   double *const *out, int nthreads);

/* nsteps steps with ping-pong buffers; final state in `state` */
void orc_run(const orc_grid *g, const orc_velocity *vel, int trace, int cross,
             double t0, double dt, int nsteps, double *const *state,
             double *const *scratch, int nthreads);

/* diagnostics (Sec. 6, eq. maximum_norm; volume by sub-sampling) */
double orc_emax(long n, const double *a, const double *b);
/* measure (area/volume) of {H < 0}: q^p cell-centred samples per cell */
double orc_measure_negative(const orc_grid *g, const double *const *planes, int q,
                            int nthreads);
/* measure of the symmetric difference {H_a < 0} xor {H_b < 0}, same sampling;
 * also counts samples where |H_a| < eps (sign decision close to rounding) */
double orc_symdiff(const orc_grid *g, const double *const *a, const double *const *b,
                   int q, double eps, long *n_ambiguous, int nthreads);
/* Hermite value and gradient at arbitrary points (cell located by floor+clamp) */
void orc_eval_points(const orc_grid *g, const double *const *planes, long npts,
                     const double *pts, double *H, double *grad);

/* Normal and curvature at arbitrary points from the interpolant of the cell holding
 * each point (Sec. 3.4): n = grad H / |grad H| (eq. surface_normal); in 2D
 * kappa = (H_xx H_y^2 - 2 H_x H_y H_xy + H_yy H_x^2) / |grad H|^3 (eq. curvature), in 3D
 * its extension kappa = div(grad H / |grad H|) = (|g|^2 tr(D^2 H) - g^T D^2 H g) / |g|^3,
 * g = grad H (the sum of the principal curvatures; the 2D formula is its p = 2 case).
 * Where grad H = 0, n = 0 and kappa = 0.  H[npts], normal[npts*dim], kappa[npts]. */
void orc_curvature_points(const orc_grid *g, const double *const *planes, long npts,
                          const double *pts, double *H, double *normal, double *kappa);

#ifdef __cplusplus
}
#endif
#endif
