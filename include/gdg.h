/*
 * gdg.h -- C ABI of the GB300 energy-based DG / Galerkin-difference library.
 *
 * The library advances the second-order wave equation
 *     u_t = v,   v_t = div(c^2 grad u)                       (Section 2, Eqs. 1-2)
 * discretised by the energy-based DG method on tensor-product elements with
 * the Galerkin-difference (GD) basis of degree p (odd) on N cells per element
 * per direction (Section 2.1), interelement fluxes of Section 2.2.1, and
 * classic RK4 in time (Sections 3.3, 6).
 *
 * Conventions for every call
 *   - Return value: GDG_OK (0) or a negative GDG_E* status.  No call aborts
 *     or exits; after GDG_ECUDA the CUDA error text is in gdg_last_error().
 *   - "device" pointers are CUDA global-memory addresses on the context's
 *     device, owned by the caller (e.g. torch tensors); "host" pointers are
 *     ordinary process memory, also caller-owned.  Nothing is retained after
 *     a call returns except what gdg_create copies.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on that stream unless they return a
 *     host value (gdg_energy, gdg_pcg statistics, gdg_step_host).
 *   - A context is not thread-safe; use one context per stream at a time.
 *   - Nodal layout of a field (doubles): 1-D u[e*n1 + i];
 *     2-D u[((ey*nx + ex)*n1 + j)*n1 + i], i along x (fastest), n1 = N+1,
 *     value at the GD node (x_e + i*Hx/N, y_e + j*Hy/N).  Element interface
 *     nodes are duplicated (the method is discontinuous between elements).
 */
#ifndef GDG_H
#define GDG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define GDG_OK           0
#define GDG_EINVAL      -1   /* bad argument: even p, p > N, null pointer, bad enum, size mismatch */
#define GDG_ENOMEM      -2   /* device or host allocation failed                                */
#define GDG_ECUDA       -3   /* CUDA runtime error (text in gdg_last_error)                      */
#define GDG_ENOCONV     -4   /* PCG hit pcg_maxit; result = last iterate, statistics filled      */
#define GDG_ETIMEOUT    -5   /* a bounded device-side wait gave up                               */
#define GDG_ENONFINITE  -6   /* NaN or Inf detected (energy, PCG residual)                       */
#define GDG_EUNSUPPORTED -7  /* valid request the library does not provide (e.g. N+1 > 16)       */
#define GDG_EHALO       -8   /* the caller's halo exchange function reported a failure            */

/* ---- enums ----------------------------------------------------------- */
enum { GDG_BC_DIRICHLET = 0, GDG_BC_PERIODIC = 1 };
/* Section 2.2.1: central alpha=1/2, beta=tau=0; upwind alpha=1/2, beta=xi/2,
 * tau=1/(2 xi); alternating alpha=1, beta=tau=0, with the sides of a face
 * labelled by a fixed orientation (side 1 = the left / lower element, so
 * v* = v_left and (grad u)* = grad u_right on every interior face) and the
 * closure v* = 0, (n.grad u)* = n.grad u_in on a Dirichlet side. */
enum { GDG_FLUX_CENTRAL = 0, GDG_FLUX_UPWIND = 1, GDG_FLUX_ALTERNATING = 2 };
/* Coefficients: constant c^2 on a Cartesian box mesh, or c^2 and the element
 * geometry sampled at every element's GD nodes (Section 7: variable speed of
 * sound or mapped, non-Cartesian elements). */
enum { GDG_COEF_CONST = 0, GDG_COEF_NODAL = 1 };
/* Local solves: modified-basis diagonalisation (Section 3.2, constant
 * coefficient Cartesian only), element-local preconditioned CG (Section
 * 7.1), or precomputed element inverses (GDG_COEF_NODAL only): the
 * precomputed-inverse route that Section 3.1 discusses, applied to the
 * time-independent element systems of Section 7.1.  gdg_create forms
 * (S_c2 + w w^T)^-1 and M_J^-1 per element by Cholesky and folds them with
 * the face lifts and the stiffness matrix into G_u = (S_c2 + w w^T)^-1 R_u,
 * G_v = M_J^-1 R_v and K = M_J^-1 S_c2 (R_u, R_v: the lifts of the face line
 * integrals into r_u, r_v; (12 (N+1) + (N+1)^2) (N+1)^2 more doubles per
 * element are kept, the inverses are freed after setup); every stage then
 * applies them instead of running PCG.  FP64 only (GDG_EUNSUPPORTED with
 * GDG_MIXED); gdg_pcg still runs PCG on such a context. */
enum { GDG_SOLVE_DIAG = 0, GDG_SOLVE_PCG = 1, GDG_SOLVE_INVERSE = 2 };
/* PCG preconditioner: frozen-coefficient diagonalisation, none (plain CG),
 * or the zero fill-in incomplete Cholesky factors of Section 7.1, which the
 * library does not run on the GPU (their triangular solves are sequential per
 * element; gdg_create returns GDG_EUNSUPPORTED). */
enum { GDG_PC_FDM = 0, GDG_PC_NONE = 1, GDG_PC_IC0 = 2 };
/* Arithmetic of the element solves.  GDG_FP64 everywhere, or (GDG_SOLVE_PCG
 * only) FP32 inner PCG with FP64 iterative refinement of every solve (FP64
 * state, residuals, lifts, norms and energy; same FP64 stopping test).
 * Constant-coefficient contexts are FP64 only (GDG_EUNSUPPORTED otherwise):
 * their diagonal solves have no iteration to refine. */
enum { GDG_FP64 = 0, GDG_MIXED = 1 };
/* Inner solves in TF32 or BF16 (GDG_EUNSUPPORTED): refinement converges at
 * about kappa u_low per sweep and the u_t element systems have kappa ~ 1e3
 * to 1e5, so these need several times the FP64 sweeps of GDG_MIXED (whose
 * inner solves are FP32) or do not converge. */
enum { GDG_TF32 = 2, GDG_BF16 = 3 };
/* State representation used inside gdg_step for the diagonalised route:
 * GDG_ROUTE_MODAL keeps the modal coefficients U = Psi Ubar (Section 3.2)
 * from the first stage to the last; GDG_ROUTE_NODAL keeps the nodal state
 * and transforms every stage's input to the modal basis and its k back
 * (two n1 x n1 contractions per direction and field each way), combining
 * the RK stages on nodal vectors.  Both give the same U', V' to rounding;
 * the nodal route does four separable transforms more per stage.  Nodal:
 * dim 1 and 2, whole meshes (GDG_EUNSUPPORTED otherwise). */
enum { GDG_ROUTE_MODAL = 0, GDG_ROUTE_NODAL = 1 };
/* Operator selector of gdg_mass_solve / gdg_pcg. */
enum { GDG_OP_M = 0, GDG_OP_S = 1 };

typedef struct gdg_ctx gdg_ctx;   /* opaque; owns uploaded operators and scratch */

typedef struct {
    int dim;             /* 1, 2 or 3 (3: GDG_COEF_CONST only, N+1 <= 10)           */
    int n_elem[3];       /* elements per direction (n); entries >= dim ignored       */
    int N;               /* GD cells per element per direction, n1 = N+1 <= 16       */
    int p;               /* odd GD degree, 1 <= p <= N                               */
    double lo[3], hi[3]; /* box [lo, hi] of the (reference) mesh                     */
    int bc[3];           /* per direction: GDG_BC_DIRICHLET (u = 0) or _PERIODIC     */
    int flux;            /* GDG_FLUX_*                                               */
    double xi;           /* upwind splitting; <= 0 means xi = c (local c for NODAL)  */
    int coef;            /* GDG_COEF_*                                               */
    double c2;           /* constant c^2 (GDG_COEF_CONST)                            */
    const double *x_nodes;  /* host, GDG_COEF_NODAL (2-D): physical x at every      */
    const double *y_nodes;  /*   element node, nodal layout; copied by gdg_create    */
    const double *c2_nodes; /* host, GDG_COEF_NODAL: c^2 at every element node       */
    int nquad;           /* Gauss points per GD cell per direction (0: p+1)          */
    int solver;          /* GDG_SOLVE_* (GDG_COEF_NODAL requires GDG_SOLVE_PCG)      */
    int precond;         /* GDG_PC_*                                                 */
    double pcg_rtol;     /* stop when ||r||_2 <= rtol ||b||_2 per element system     */
    int pcg_maxit;       /* iteration cap per element system                         */
    int precision;       /* GDG_FP64 or GDG_MIXED                                    */
    int route;           /* GDG_ROUTE_* (diagonalised route only)                    */
    int refine_max;      /* GDG_MIXED: maximum FP64 refinement sweeps per solve      */
    double refine_rtol;  /* GDG_MIXED: inner FP32 PCG relative tolerance             */
    int rows[2];         /* 2-D GDG_COEF_CONST: the element rows [rows[0], rows[1])  */
                         /* of the n_elem[1]-row mesh this context owns (a band of   */
                         /* an element-partitioned mesh, see gdg_set_halo); {0, 0}   */
                         /* = every row.  A band that does not start at row 0 or end */
                         /* at the last row has a halo side there; bc[1] must then  */
                         /* be GDG_BC_DIRICHLET (it applies to the mesh's own sides) */
} gdg_problem;

typedef struct {
    int max_iters;        /* largest per-element PCG iteration count (FP32 inner    */
                          /* iterations summed over sweeps under GDG_MIXED)         */
    double mean_iters;    /* mean over elements                                    */
    double max_rel_resid; /* largest final ||r||/||b|| (true FP64 residual)        */
    int unconverged;      /* element systems that hit pcg_maxit (GDG_MIXED:        */
                          /* refine_max) above pcg_rtol                             */
    int max_sweeps;       /* GDG_MIXED: largest number of FP64 refinement sweeps   */
    double mean_sweeps;   /* GDG_MIXED: mean sweeps (FP64 residuals after the first) */
    long long guessed;    /* u_t solves started from the learned guess (gdg_mlp_attach) */
    long long fell_back;  /* ... of which restarted from 0 (guess no better than 0)   */
} gdg_pcg_stats;

/* Human-readable text of a status code (static storage). */
const char *gdg_status_string(int status);

/* Text of the last error recorded on ctx ("" if none). */
const char *gdg_last_error(const gdg_ctx *ctx);

/*
 * 1-D GD basis on the reference element [0,1] (host only; Sections 2.1, 2.1.1,
 * 3.1, 3.2).  Nodes r_i = i/N; on cell k the basis is the Lagrange basis of
 * the p+1 nodes starting at s(k) = min(max(k-q+1, 0), N-p), q = (p+1)/2,
 * which is the GD basis with the extrapolation boundary modification.
 * Outputs (caller-owned host arrays, row-major, any may be NULL):
 *   M, S [n1*n1]  mass int phi_k phi_l and stiffness int phi_k' phi_l'
 *   phiL, phiR [n1]  basis values at r = 0 and r = 1
 *   dphiL, dphiR [n1]  one-sided derivatives at r = 0 and r = 1
 *   Psi [n1*n1], lambda [n1]  S Psi = M Psi diag(lambda), Psi^T M Psi = I,
 *                     lambda ascending with lambda[0] = 0 (constant mode),
 *                     Psi[i*n1 + k] = component i of eigenvector k.
 * Errors: GDG_EINVAL for even p, p < 1, N < p; GDG_EUNSUPPORTED for N+1 > 16.
 */
int gdg_basis_1d(int p, int N, double *M, double *S, double *phiL, double *phiR,
                 double *dphiL, double *dphiR, double *Psi, double *lambda);

/*
 * Validate *pb, build the element operators on the host (basis, Kronecker
 * factors and modified basis for GDG_COEF_CONST; quadrature assembly of
 * the element mass and stiffness matrices and face data on the device for
 * GDG_COEF_NODAL, Section 7.1) and allocate device scratch on the current
 * CUDA device.  Host arrays in *pb are copied.  *out receives the context.
 * GDG_COEF_NODAL also builds, per element face, the linear map from the
 * element's and the neighbour's face lines (v, normal slope, u along the
 * face; 3 (N+1) values each) to the lifted face integrals: the traces at
 * the face quadrature points, the flux of Section 2.2.1 and the integrals
 * against the face basis, all fixed in time (72 (N+1)^2 doubles per
 * element); elements then exchange face lines instead of point traces.
 * Nodal layout of the state: 1-D u[e*n1 + i]; 2-D u[(e*n1 + j)*n1 + i],
 * e = ey*nx + ex; 3-D u[((e*n1 + k)*n1 + j)*n1 + i], e = (ez*ny + ey)*nx + ex
 * (i along x; element nodes on shared faces are duplicated, as in DG).
 * Errors: GDG_EINVAL, GDG_EUNSUPPORTED (e.g. 3-D with GDG_COEF_NODAL or
 * N+1 > 10), GDG_ENOMEM, GDG_ECUDA.
 */
int gdg_create(const gdg_problem *pb, gdg_ctx **out);

/* Free the context and its device memory (synchronises the device). */
int gdg_destroy(gdg_ctx *ctx);

/* Doubles per field: n^d * (N+1)^d (the paper's DOF count, Section 3.3). */
long long gdg_state_len(const gdg_ctx *ctx);

/*
 * Semi-discrete time derivative (Eqs. DG1, DG2, DG1_extra with the fluxes of
 * Section 2.2.1): du = dU/dt, dv = dV/dt at the nodal state (u, v) and time
 * t (t enters only through a point source, gdg_set_point_source; the
 * problem is otherwise autonomous).  Device pointers of gdg_state_len
 * doubles; du, dv must not alias u, v.  GDG_SOLVE_PCG contexts use the PCG
 * settings of the problem and may return GDG_ENOCONV (results are then the
 * last iterates).
 */
int gdg_rhs(gdg_ctx *ctx, const double *u, const double *v, double t, double *du, double *dv,
            void *stream);

/*
 * Element-local solve with the diagonalised operators (Section 3.2):
 *   which = GDG_OP_M:  x = M^-1 b               (M = Psi^-T Psi^-1)
 *   which = GDG_OP_S:  S x = b, w^T x = 0, w = M 1 (the u_t system of
 *                      Eq. DG1 with Eq. DG1_extra; b must satisfy 1^T b = 0
 *                      per element, as every r_u does)
 * b, x: device, gdg_state_len doubles, nodal layout; may alias.
 * GDG_COEF_CONST contexts only (GDG_EINVAL otherwise; use gdg_pcg).
 */
int gdg_mass_solve(gdg_ctx *ctx, int which, const double *b, double *x, void *stream);

/*
 * Element-local preconditioned CG (Section 7.1) on every element's system
 *   which = GDG_OP_M:  M_J x = b
 *   which = GDG_OP_S:  (S_c2 + w w^T) x = b, w = M_J 1 / |e|, |e| = 1^T M_J 1
 *                      the element area (the SPD form of the constrained u_t
 *                      system: for 1^T b = 0 its solution has S_c2 x = b,
 *                      w^T x = 0; the 1/|e| weight keeps the rank-one term O(1))
 * x is the initial guess on entry and the solution on exit (device).
 * Stops per element when ||r||_2 <= pcg_rtol ||b||_2 or after pcg_maxit
 * iterations.  stats (host, may be NULL) is filled; the call synchronises
 * stream when stats != NULL.  GDG_ENOCONV if any element hit pcg_maxit.
 * GDG_COEF_NODAL contexts only.
 */
int gdg_pcg(gdg_ctx *ctx, int which, const double *b, double *x, gdg_pcg_stats *stats,
            void *stream);

/*
 * PCG iteration statistics of the element solves done inside gdg_step and
 * gdg_rhs on a GDG_SOLVE_PCG context since the previous call, for the u_t
 * system (u_sys) and the v_t system (v_sys); either may be NULL.  Resets the
 * counters.  mean_iters is per element solve; max_rel_resid is not tracked
 * here (0).  Synchronises the device.  GDG_EINVAL on GDG_COEF_CONST contexts.
 */
int gdg_step_stats(gdg_ctx *ctx, gdg_pcg_stats *u_sys, gdg_pcg_stats *v_sys);

/*
 * Advance (u, v) in place by nsteps classic RK4 steps of size dt starting at
 * t0 (device pointers; t0 matters only with a point source).  The per-stage
 * work is the whole hot path: traces,
 * fluxes and lifts, stiffness, constrained u_t solve, mass inversion and the
 * stage combination.  Launches are captured in a CUDA graph on first use.
 */
int gdg_step(gdg_ctx *ctx, double *u, double *v, double t0, double dt, int nsteps,
             void *stream);

/*
 * gdg_step on HOST arrays: copies (u, v) to the device, advances nsteps and
 * copies the result back, all on stream, and synchronises before returning.
 * u, v: host, gdg_state_len doubles each (pinned memory makes the copies
 * asynchronous DMA; pageable memory works but is slower).
 */
int gdg_step_host(gdg_ctx *ctx, double *u, double *v, double t0, double dt, int nsteps,
                  void *stream);

/*
 * Stage kernel of a 2-D constant-coefficient context (the modal route of
 * Section 3.2; not a method choice, a launch choice): 0 = one thread per
 * element line, 1 = two threads per line (even / odd modes), 2 = one thread
 * per line and field (u and v in separate warps), 3 = all stages of a
 * gdg_step call in one persistent cooperative launch (each line's state in
 * registers, each block synchronised with the blocks holding its face
 * neighbours between stages; only for N+1 <= 10 and where every block of
 * the grid fits the GPU at once, GDG_EUNSUPPORTED otherwise), -1 = choose by
 * timing all eligible variants at the next gdg_step (the default).  All
 * variants perform the same floating-point operations in the same order:
 * results are bit-identical.  Setting a variant drops any captured step
 * graph.  Under variant 3 gdg_step synchronises its stream at the end (to
 * read the give-up flag of its waits) and returns GDG_ETIMEOUT if a wait
 * lasted longer than the wait limit (the state is then invalid; the
 * context stays usable).
 * GDG_EINVAL on other contexts or values; get: the variant in use (-1 before
 * the choice is made).
 */
int gdg_set_stage_variant(gdg_ctx *ctx, int variant);
int gdg_get_stage_variant(const gdg_ctx *ctx, int *variant);

/*
 * Bound on any device-side wait of ctx's kernels (the persistent step's
 * waits for neighbouring blocks between stages), in seconds of wall time;
 * default 1.  A wait that runs out sets a flag, every block leaves the
 * kernel, and the call returns GDG_ETIMEOUT.  GDG_EINVAL for seconds <= 0
 * or not finite.
 */
int gdg_set_wait_limit(gdg_ctx *ctx, double seconds);

/*
 * Discrete energy E = 1/2 sum_e (V_e^T M_e V_e + U_e^T S_e U_e) with S_e the
 * c^2-weighted stiffness (Section 6's energy norm squared, halved).
 * u, v device; *E host; synchronises stream.  GDG_ENONFINITE if E is not finite.
 */
int gdg_energy(gdg_ctx *ctx, const double *u, const double *v, double *E, void *stream);

/*
 * Element residuals of the semi-discretisation before the local solves
 * (Eqs. DG1, DG2 with the fluxes of Section 2.2.1, Section 7.1 quadrature):
 *   ru = sum_faces int c^2 (n.grad phi)(v* - v),  rv = -S_c2 u + sum_faces int c^2 phi q*
 * so that (S_c2 + w w^T)(du - v) = ru and M_J dv = rv.  Device arrays,
 * nodal layout.  GDG_COEF_NODAL contexts only.
 */
int gdg_residuals(gdg_ctx *ctx, const double *u, const double *v, double *ru, double *rv, void *stream);

/*
 * Point source (the forcing f of u_tt = div(c^2 grad u) + f):
 *   f(x, t) = amplitude sin(omega t) delta(x - x_s)
 * on a GDG_COEF_NODAL context.  x_s is given by the element holding it and
 * its reference coordinates (r, s) in [0,1]^2 (the point of the element's
 * isoparametric map; on a Cartesian mesh x = x_e + r H_x, y = y_e + s H_y).
 * Its load on r_v is int phi_a f = phi_a(r, s) amplitude sin(omega t) on
 * that element (the delta function makes the Jacobian drop out); the inverse
 * route adds M_J^-1 of it to dV/dt.  gdg_step evaluates the source at each
 * RK stage's time, starting from its t0; gdg_rhs at its own t; gdg_residuals
 * at the time the last gdg_step reached or gdg_rhs used (0 before any).  amplitude = 0 removes the
 * source.  Drops any captured step graph; synchronises the device.
 * GDG_EINVAL: not a GDG_COEF_NODAL context, element out of range, (r, s)
 * outside [0,1]^2, non-finite amplitude or omega.
 */
int gdg_set_point_source(gdg_ctx *ctx, int element, double r, double s, double amplitude, double omega);

/* ---- element-partitioned meshes (one mesh over several contexts) ------- */
/*
 * Elements interact only through the fluxes of their shared faces (Section
 * 2.2, Eqs. DG1-DG2 are element-local apart from the face terms of Section
 * 2.2.1), so one 2-D constant-coefficient mesh can be split by rows of
 * elements over several contexts (typically one per GPU): each context owns
 * a contiguous band of element rows and, before every RK stage, needs the
 * traces (v and n.grad u along the face, N+1 modal values each) of the
 * facing row of its neighbours.  A context whose problem owns a band of
 * rows (rows[] set, every other field as for the whole mesh, so that every
 * band computes the same element operators) with a neighbour band below or
 * above packs its boundary row's traces into send buffers, calls the
 * caller's exchange function, and unpacks the neighbours' traces from the
 * receive buffers, once at the start of gdg_step / gdg_rhs and after every
 * stage but the last of a gdg_step call.
 *
 * gdg_halo_len: doubles in one side's buffer, n_elem[0] * 2 * (N+1)
 *   (layout [ex][v | n.grad u][mode]), -1 for a context without halo sides.
 * gdg_set_halo: register the caller-owned device buffers of both sides
 *   (send_lo / recv_lo for the lower side, send_hi / recv_hi for the upper;
 *   NULL for a side without a halo) and the exchange function.
 *   fn(user, stream) is called on the host, in stream order, after the
 *   send buffers' pack kernel has been enqueued on `stream` (the cudaStream_t
 *   of the gdg_step / gdg_rhs call, as void*); it must make the neighbour
 *   below's send_hi arrive in recv_lo and the neighbour above's send_lo in
 *   recv_hi before later work on `stream` reads them (for example by
 *   stream-ordered NCCL send / receive, or by synchronising, copying through
 *   host memory and copying back), and return 0, or nonzero on failure
 *   (the call then returns GDG_EHALO).  Contexts with a halo side launch
 *   their stages directly (no CUDA graph, no persistent step: stage variant
 *   0).  gdg_energy of such a context sums its own elements only.
 * Errors: GDG_EINVAL (no halo side, a buffer missing for a halo side, fn NULL).
 */
typedef int (*gdg_halo_fn)(void *user, void *stream);
long long gdg_halo_len(const gdg_ctx *ctx);
int gdg_set_halo(gdg_ctx *ctx, double *send_lo, double *send_hi, double *recv_lo, double *recv_hi,
                 gdg_halo_fn fn, void *user);

/* ---- learned initial guess for the u_t solve (not in the paper) -------- */
/*
 * A three-layer perceptron 162 -> 64 -> 64 -> 81 (tanh, tanh, linear) maps an
 * element's features x = [c^2/mean(c^2) at its 81 nodes, r_u/||r_u||] to a
 * guess of y/||r_u|| for (S_c2 + w w^T) y = r_u; the PCG of the u_t system
 * then starts from ||r_u|| * guess, or from 0 when the guess's true FP64
 * residual is not smaller than ||r_u|| (plain PCG is the fallback).
 * Parameters: an FP32 master block params[GDG_MLP_NPARAM] in the order
 *   W1[64][162], b1[64], W2[64][64], b2[64], W3[81][64], b3[81]
 * and BF16 working weights w_bf16[GDG_MLP_NWEIGHT] = W1, W2, W3 (uint16_t
 * bit patterns); the kernels multiply in FP32 with BF16 weights.
 * All pointers below are device pointers unless stated.
 */
#define GDG_MLP_IN 162
#define GDG_MLP_HID 64
#define GDG_MLP_OUT 81
#define GDG_MLP_NPARAM 19857
#define GDG_MLP_NWEIGHT 19648

/* Y[B][81] = net(X[B][162]). */
int gdg_mlp_forward(const uint16_t *w_bf16, const float *params, const float *X, int B, float *Y,
                    void *stream);

/* Floats of the per-CTA partial buffer gdg_mlp_backward needs for B samples. */
long long gdg_mlp_partial_len(int B);

/*
 * Mean-squared loss L = (1/B) sum_s ||net(X[idx[s]]) - T[idx[s]]||^2 over the
 * B samples idx[0..B) (idx NULL: the first B rows) and its gradient
 * grad[GDG_MLP_NPARAM] (same order as params); *loss on the device.
 * partial: gdg_mlp_partial_len(B) floats of scratch.  Deterministic.
 */
int gdg_mlp_backward(const uint16_t *w_bf16, const float *params, const float *X, const float *T,
                     const int *idx, int B, float *partial, float *grad, float *loss, void *stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8; step counts from 1) on params,
 * with moment buffers m, v, then refresh of w_bf16 (round to nearest even). */
int gdg_mlp_adam(float *params, float *m, float *v, const float *grad, int step, float lr, uint16_t *w_bf16,
                 void *stream);

/* w_bf16 = BF16(weights of params). */
int gdg_mlp_to_bf16(const float *params, uint16_t *w_bf16, void *stream);

/*
 * Training rows of every element of a GDG_COEF_NODAL context from a residual
 * ru (e.g. of gdg_residuals): X[ne][162] features and, when y is not NULL
 * (the u_t solution, e.g. from gdg_pcg), T[ne][81] = y/||r_u||.
 */
int gdg_mlp_rows(gdg_ctx *ctx, const double *ru, const double *y, float *X, float *T, void *stream);

/* Use (copies of) the network in every u_t solve of gdg_step / gdg_rhs on ctx. */
int gdg_mlp_attach(gdg_ctx *ctx, const uint16_t *w_bf16, const float *params);

/* Back to plain PCG from x0 = 0. */
int gdg_mlp_detach(gdg_ctx *ctx);

/* ---- batches of independent problems ---------------------------------- */
typedef struct gdg_batch gdg_batch;   /* opaque; owns one context per problem */

/*
 * Many independent 2-D problems advanced together (a launch pattern layered
 * on the method; the paper advances one mesh at a time).  Every RK stage of
 * all problems is ONE persistent launch: (SMs x resident blocks) blocks of
 * one element block each (N1^2 threads rounded up to a warp) walk one list
 * of work items ordered longest first -- the element solves of the
 * GDG_COEF_NODAL problems (each with its own solver and precision: element
 * PCG in FP64 or GDG_MIXED, or precomputed inverses), then tiles of the
 * GDG_COEF_CONST problems' elements (modified-basis route) -- block b taking
 * turns b, b + G, ... of a few consecutive items.  A call's launches are
 * replayed from one CUDA
 * graph.  The kernel's register budget (three compiled variants) and the
 * resident blocks per SM are chosen on the first gdg_batch_step by timing
 * the candidates on the batch's own data.
 * pbs[count]: host problems, all dim = 2 with the same N, 7 <= N <= 9, whole
 * meshes (rows = {0, 0}); each is validated and set up as by gdg_create (host
 * arrays copied).
 * Errors: as gdg_create; GDG_EUNSUPPORTED for other N or bands of rows.
 */
int gdg_batch_create(const gdg_problem *pbs, int count, gdg_batch **out);

/* Free the batch and its contexts (synchronises the device). */
int gdg_batch_destroy(gdg_batch *b);

/* Doubles per field of problem i (as gdg_state_len), -1 on bad arguments. */
long long gdg_batch_state_len(const gdg_batch *b, int i);

/*
 * Advance every problem i in place by nsteps RK4 steps of size dt[i].
 * u, v: host arrays of count device pointers (problem i's nodal state,
 * gdg_batch_state_len doubles each); dt: host array of count step sizes.
 * Each problem's result equals its own gdg_step with the same settings.
 */
int gdg_batch_step(gdg_batch *b, double *const *u, double *const *v, const double *dt, int nsteps,
                   void *stream);

/*
 * Launch shape chosen by the tuner (zeros before the first gdg_batch_step;
 * any output pointer may be NULL): threads_per_block of the stage launch
 * (N1^2 rounded up to a warp), blocks_per_sm (the persistent grid has SMs x
 * blocks_per_sm blocks), tile_elements = threads_per_block / (2 N1), the
 * elements of a constant-coefficient work item (0 when the batch has none),
 * register_budget (see gdg_batch_set_tuning) and registers_per_thread of the
 * chosen kernel, items_per_turn (block b takes the turns b, b + G, ... of
 * that many consecutive items of the list).
 */
int gdg_batch_tuning(const gdg_batch *b, int *threads_per_block, int *blocks_per_sm, int *tile_elements,
                     int *register_budget, int *registers_per_thread, int *items_per_turn);

/*
 * Pin the launch shape instead of tuning it: register_budget 0, 1 or 2 (the
 * kernel compiled for 3 resident blocks of N1^2 threads per SM, for 480
 * threads per SM (at most 128 registers a thread) or for 960 (at most 64)),
 * blocks_per_sm >= 1 (the persistent grid has SMs x blocks_per_sm blocks),
 * items_per_turn >= 1; blocks_per_sm = 0 hands the choice back to the tuner
 * at the next gdg_batch_step.  Synchronises the device.
 * Errors: GDG_EINVAL for other values or more blocks per SM than the
 * kernel's registers and the batch's shared memory allow.
 */
int gdg_batch_set_tuning(gdg_batch *b, int register_budget, int blocks_per_sm, int items_per_turn);

/* PCG statistics of problem i since the previous call, as gdg_step_stats. */
int gdg_batch_stats(gdg_batch *b, int i, gdg_pcg_stats *u_sys, gdg_pcg_stats *v_sys);

/*
 * gdg_rhs_static -- the semi-discrete time derivative of gdg_rhs for a
 * constant-coefficient Cartesian problem (GDG_COEF_CONST), computed without
 * allocating anything.  The paper has no counterpart to this call.
 *
 * Who it is for: callers that cannot call cudaMalloc -- for example a plug-in
 * inside a host application whose own memory pool already holds all free
 * device memory (a fresh cudaMalloc would fail although the application has
 * room), or a control loop that cannot afford the device-wide
 * synchronisation cudaMalloc may perform.  Such callers cannot create a
 * gdg_ctx either (gdg_create allocates), so this call takes the problem
 * itself: the basis and modal tables are rebuilt on the host in fixed-size
 * stack arrays on every call, and every device-side intermediate (tables,
 * modal state, modal derivative, face traces) lives in one static device
 * array of 2,097,152 doubles (16 MiB) that the library reserves on every GPU
 * that loads it, until the process exits.
 *
 * pb: host problem, only GDG_COEF_CONST.  u, v, du, dv: device, nodal layout,
 * n^d (N+1)^d doubles each; du, dv must not alias u, v.  Same result as
 * gdg_rhs on a context created from *pb (to rounding).
 * Size limit: 6 n1^2 + 2 n1^d + (4 n1^d + T) n^d doubles must fit the array,
 * with n1 = N+1 and T = 8 n1 (2-D) or 4 (1-D) trace words per element
 * (2-D, N = 8: up to 5,294 elements, e.g. 72 x 72); larger meshes return
 * GDG_EUNSUPPORTED with a message on stderr.
 * Set-up: the first call on each device, with that device current, looks up
 * the array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.
 * Sharing: every call writes each part of the array before reading it, so
 * nothing carries over between calls, but all calls on a device share the
 * one array: calls that overlap on the GPU (different streams or host
 * threads) race and corrupt each other's results.
 * Errors: GDG_EINVAL (bad problem or pointers), GDG_EUNSUPPORTED (too large,
 * N+1 > 16), GDG_ECUDA (no text is kept: there is no context).
 */
int gdg_rhs_static(const gdg_problem *pb, const double *u, const double *v, double *du, double *dv,
                   void *stream);

/* ---- kernel timing (measurement support; not part of the method) ------ */
/*
 * FP64 throughput probe: one launch, on stream, of a kernel in which every
 * thread of a grid that fills every SM runs 8 independent chains of
 * x <- x a + b FP64 fused multiply-adds, 4 per chain for each of `iters`
 * iterations (no memory
 * traffic inside the loop).  *flops (host) receives the launch's flop count
 * (an FMA counts 2); the caller times the launch (e.g. CUDA events on the
 * same stream) to obtain the FP64 rate the GPU sustains, the peak against
 * which the FP64-bound kernels of this library are compared.  sink: device
 * pointer to one double (written).  GDG_EINVAL for iters < 1 or null pointers.
 */
int gdg_probe_fp64(int iters, double *sink, double *flops, void *stream);

/* ---- index checks of the debug build ---------------------------------- */
/*
 * The library built with -DGDG_CHECKS=1 (libgdg_checks.so, build.build(checks=True);
 * the binding loads it when the environment has GDG_CHECKS=1) checks every
 * element index a kernel derives from another one: the face neighbours of
 * the stage kernels (1-D, 2-D, 3-D, variable coefficients), the neighbour
 * blocks of the persistent step and the work items of the batched launch.
 * A failed check does not trap: it is counted, the first one is recorded
 * (site, index, violated bound) and the index is replaced by a valid one, so
 * the kernel completes with a wrong result and the host reads the record.
 *
 * gdg_check_status: synchronises the device, returns the failures since the
 * last reset (count, and site / index / bound of the first one; any pointer
 * may be NULL) and, with reset != 0, zeroes them.  Sites: 1-4 one-line 2-D
 * modal body, 5-8 half-line body, 9-12 generic 2-D stage, 13-16 field-split
 * stage, 17-20 persistent step (x-, x+, y-, y+), 21 persistent step's
 * neighbour block, 22-23 1-D stage, 30-35 3-D stages (x-, x+, y-, y+, z-, z+),
 * 40 variable-coefficient face neighbour, 50 batched item's problem, 51
 * batched item's element or tile, 99 self-test.
 * gdg_check_selftest: checks `index` against [0, bound) in a one-thread
 * kernel on `stream` (a failing pair records site 99): the recording path
 * itself, without an out-of-range access anywhere.
 * Errors: GDG_EUNSUPPORTED in the ordinary build (outputs zeroed).
 */
int gdg_check_status(long long *count, int *site, long long *index, long long *bound, int reset);
int gdg_check_selftest(long long index, long long bound, void *stream);

/* Kernel kinds reported by gdg_profile_read. */
enum {
    GDG_K_STAGE = 0,      /* fused RK-stage kernel (fluxes, lifts, solves, combine, traces) */
    GDG_K_TRACES = 1,     /* trace kernel at the start of gdg_step / gdg_rhs             */
    GDG_K_TRANSFORM = 2,  /* nodal <-> modal element transforms                          */
    GDG_K_RHS = 3,        /* variable-coefficient residual kernel                         */
    GDG_K_PCG = 4,        /* element-local PCG kernel                                     */
    GDG_K_OTHER = 5,
    GDG_K_COUNT = 6
};

/*
 * on != 0: subsequent gdg_step / gdg_rhs calls on ctx launch without the
 * CUDA graph and bracket every kernel with CUDA events on the caller's
 * stream (adds a little host overhead per launch); on == 0 restores graph
 * launches.  Enabling also clears the accumulated records.
 */
int gdg_profile_enable(gdg_ctx *ctx, int on);

/*
 * Synchronise and accumulate the recorded launches of one kernel kind:
 * *launches = number of launches, *ms = summed device time (CUDA events).
 */
int gdg_profile_read(gdg_ctx *ctx, int kind, long long *launches, double *ms);

#ifdef __cplusplus
}
#endif

#endif /* GDG_H */
