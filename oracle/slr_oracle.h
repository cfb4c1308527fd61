/*
 * FP64 CPU oracle for the semi-Lagrangian level-set step of
 * Preda & Semplice, "Surface reconstruction from point cloud using a
 * semi-Lagrangian scheme with local interpolator" (arXiv 2410.22205).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library. The product path
 * (the CUDA library and its Python binding) never calls it and shares no
 * code with it.
 *
 * Plain, slow, obviously correct: one node at a time, FP64, built with
 * -ffp-contract=off so that a*b+c is never fused. Every function cites the
 * passage of the paper it follows. Grid layout: node (i,j,k) has linear
 * index i + n0*(j + n1*k), x fastest; in 2-D n2 == 1.
 *
 * Parity pins (what fixes each function independently of this code) live in
 * tests/test_oracle_pins.py. Functions pinned only in part:
 *   or_evolve_reinit, or_reconstruct -- parity partial: end to end they are
 *                 pinned to the paper's printed circle, sphere and square
 *                 tests (Tabs. errGlobCircle, errGlobSphere, errGlobSquare)
 *                 within stated factors, not to exact values, and otherwise
 *                 through the exact pins of their parts.
 *   or_evolve  -- the paper prints no end-to-end result without the
 *                 reinitialisation; pinned through its parts (the SL step,
 *                 the band, the cut, the energy and the stop test) and a
 *                 closed form of the loop (a plane front moving toward a
 *                 line cloud by Δt per iteration).
 */
#ifndef SLR_ORACLE_H
#define SLR_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int dim;            /* 2 or 3 */
    long long n[3];     /* nodes per axis; n[2] == 1 in 2-D */
    double lo[3];       /* coordinates of node (0,0,0) */
    double h;           /* uniform mesh width Δx (§3) */
    int interp;         /* 0 = Q1 (eq. IQ1), 1 = WENO (eq. IWENO) */
    double p, delta;    /* exponent p and curvature weight δ (eq. levelset:pde) */
    double dt;          /* time step Δt */
    int band;           /* 0 = whole grid, 1 = narrow band (§3.8) */
    double gamma, beta; /* band half-width γ and cut-off inner radius β (eq. cutoff) */
    double c_sing;      /* C in the singular-gradient test |∇φ| < C Δt^α (eq. SL:2) */
    double alpha;       /* α in the same test */
    int prec;           /* 32 or 64: precision in which band membership is decided
                           and in which the cut value γ is represented */
} or_params;

/* flags reported per node by the SL update */
#define OR_FLAG_FALLBACK   1  /* singular-gradient branch (eq. SL:2) taken */
#define OR_FLAG_MARGIN     2  /* |∇φ| within 1e-6 (relative) of the singular threshold */
#define OR_FLAG_REGULAR    4  /* 3-D tangent basis regularised ((∂1φ)^2+(∂3φ)^2 == 0) */

long long or_num_nodes(const or_params* g);
void or_node_coord(const or_params* g, long long idx, double x[3]);

/* §2 / §3.4: d(x) = min_Q |x - Q| with the index of the minimiser (lowest
 * index on ties). nodes == NULL: every node, in order; else the m listed. */
void or_distance(const or_params* g, const double* pts, long long npts,
                 const long long* nodes, long long m, double* d_out, int* arg_out);

/* The same d and argmin as or_distance (identical floating-point decisions),
 * found through a k-d tree over the cloud instead of a scan of every point:
 * for clouds too large for brute force. */
void or_distance_kd(const or_params* g, const double* pts, long long npts,
                    const long long* nodes, long long m, double* d_out, int* arg_out);

/* §4 eq. dxdt: h_S, the mean over the m sampled points of the distance to
 * their nearest other point (duplicates count, at distance 0) */
double or_cloud_spacing(int dim, const double* pts, long long npts, const long long* sample, long long m);

/* §3: centred differences; one-sided first-order on the domain boundary */
void or_gradient(const or_params* g, const double* v, long long idx, double grad[3]);

/* §3.2 interpolators */
double or_interp_q1(const or_params* g, const double* v, const double x[3]);
double or_weno1d(const double v[4], double theta, double h);
double or_weno1d_weights(const double v[4], double theta, double h, double w[2]);
double or_interp_weno(const or_params* g, const double* v, const double x[3]);
double or_interp(const or_params* g, const double* v, const double x[3]);

/* §3.8 eq. cutoff, eq. subgrid, eq. cut */
double or_cutoff(const or_params* g, double u);
int or_in_band(const or_params* g, double u);
double or_cut(const or_params* g, double u);
void or_cut_all(const or_params* g, double* u);
long long or_band(const or_params* g, const double* u, long long* list_out);

/* §3.1: tangent directions */
void or_sigma2d(const double grad[3], double sigma[3]);
int or_tangent_basis(const double grad[3], double nu1[3], double nu2[3]);

/* §3.1 eq. SL2d / SL3d: feet of the characteristics of one node;
 * returns the number of feet (2 in 2-D, 4 in 3-D). ct is the scale factor
 * C^n_j already multiplied by the cut-off c(φ_j). */
int or_feet(const or_params* g, const double xj[3], const double grad_u[3], const double grad_d[3],
            double dj, double ct, double feet[4][3]);

/* scale factor C^n_j = (d_j / E_p)^(p-1) (§3.1) */
double or_scale_factor(const or_params* g, double dj, double Ep);

/* one SL update of node idx, before the cut */
double or_sl_node(const or_params* g, const double* u, const double* d, double Ep,
                  long long idx, int* flags);

/* The SL update of Algorithm 1 and the cut: u_out on every node. In band mode the nodes
 * of eq. subgrid are updated, then every node is cut (eq. cut); in whole-grid
 * mode every node is updated and nothing is cut. flags_out (may be NULL):
 * per-node flags. Returns Δ_φ = h^dim Σ |u_out - u| (§4, L1 of the update). */
double or_sl_step(const or_params* g, const double* u, const double* d, double Ep,
                  double* u_out, int* flags_out);

/* SL update (before the cut) of the m listed nodes only */
void or_sl_nodes(const or_params* g, const double* u, const double* d, double Ep,
                 const long long* nodes, long long m, double* out, int* flags);

/* §3.5 energy. out[0] = Σ |d|^p (measure) over the front, out[1] = E_p =
 * out[0]^(1/p), out[2] = the part of out[0] from 3-D subcells whose
 * |φ(x')| lies within amb_tol of the threshold (√3/2)Δx', out[3] = number
 * of front cells. R = subcells per axis (3-D only). */
void or_energy(const or_params* g, const double* u, const double* d, double p, int R,
               double amb_tol, double out[4]);

/* §4 eq. deltaEn. E2 holds E_2(φ^0..φ^n). Returns 1 to stop after n
 * iterations. *delta_out receives Δ_E^n (or -1 when not yet defined). */
int or_stop(const double* E2, int n, int kmax, double tol, int min_iters, int max_iters,
            double* delta_out);

/* Algorithm 1 loop with the stop rule of §4; u is overwritten by the final
 * state. E2_hist needs max_iters+1 entries, dphi_hist max_iters. Returns the
 * number of iterations; *converged is 1 when the Δ_E test stopped the loop. */
int or_evolve(const or_params* g, double* u, const double* d, int R, double stop_tol, int kmax,
              int min_iters, int max_iters, double* E2_hist, double* dphi_hist, int* converged);

/* §3.7 reinitialisation on Ḡ (the band {|phi_band| < γ} and its face
 * neighbours) of phi_tilde, then eq. cut; see the readings in slr_oracle.c.
 * sweeps <= 0: or_reinit_sweeps(g); dtau <= 0: h/2. out: every node.
 * flags_out (may be NULL): bit 0 in Ḡ, bit 1 interface node. Returns |Ḡ|. */
long long or_reinit(const or_params* g, const double* phi_band, const double* phi_tilde, int sweeps, double dtau,
                    double* out, unsigned char* flags_out);
int or_reinit_sweeps(const or_params* g);

/* or_evolve with the reinitialisation of Algorithm 1 (reinit != 0): after each SL step and
 * cut, or_reinit with the step's band; Δ_φ then covers the whole update. */
int or_evolve_reinit(const or_params* g, double* u, const double* d, int R, double stop_tol, int kmax,
                     int min_iters, int max_iters, int reinit, int sweeps, double dtau, double* E2_hist,
                     double* dphi_hist, int* converged);

/* §3.6 initial data: external marking from the grid boundary through nodes
 * with d >= gamma_s, φ0 = d - gamma_s there, fast sweeping of |∇φ| = 1 on
 * the other nodes, whose sign is then reversed (readings in slr_oracle.c).
 * out: every node; ext_out (may be NULL): 1 on external nodes. Returns the
 * number of external nodes. */
long long or_init_marking(const or_params* g, const double* d, double gamma_s, double* out, unsigned char* ext_out);
/* the Godunov local solution of |∇φ| = 1 used by the sweeps, from the m
 * per-axis upwind values a[0..m) (m = 1..3) */
double or_fsm_solve(const double* a, int m, double h);

/* §3.4 distance grid as the paper builds it: exact on the 4^dim node box
 * around each point, fast sweeping elsewhere; returns the box node count */
long long or_distance_fsm(const or_params* g, const double* pts, long long npts, double* d_out,
                          unsigned char* fixed_out);

/* splitmix64 (Steele, Lea and Flood 2014): the i-th output of the stream
 * started at seed (the state after i+1 increments, mixed) */
unsigned long long or_splitmix64(unsigned long long seed, unsigned long long i);

/* §4 runs from coarse to fine; see the readings in slr_oracle.c */
typedef struct {
    double h_s;
    long long sample_size;
    int runs_done;
    double run_dx[8];
    long long run_n[8][3];
    double run_lo[8][3];
    int run_iters[8];
    int run_converged[8];
    double run_energy[8];
    double run_err_cloud[8];
    double run_l1_err[8];
} or_multirun_report;
int or_reconstruct(int dim, int prec, int interp, int runs, double K_s, double sample_frac,
                   unsigned long long seed, long long max_nodes, int max_iters, int distance_fsm, int exact_sphere,
                   const double* sphere, const double* pts, long long npts, double* phi_out, long long phi_cap,
                   or_multirun_report* rep);

/* §4 L^1 error against an exact signed distance (cut at γ in band mode) */
double or_l1_error(const or_params* g, const double* u, const double* exact);
/* |x - c| - r on every node, sphere = {cx, cy, cz, r} */
void or_sdf_sphere(const or_params* g, const double* sphere, double* out);

/* nodes with |φ| < width, ascending index */
long long or_extract(const or_params* g, const double* u, double width, long long* idx_out, double* u_out);

/* §4 eq. errCloud: mean over the cloud of |I[φ](Q)| */
double or_err_cloud(const or_params* g, const double* u, const double* pts, long long npts);

/* set the OpenMP thread count used by the per-node loops (0 = library default);
 * returns the count in effect. Results do not depend on it. */
int or_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
